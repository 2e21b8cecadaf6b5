// mf_refine.cu -- objective and adjoint for gradient refinement of triggers.
// For theta = (m1, m2, t) and a fixed band [k_lo, k_hi), Eq. (1) evaluated
// directly at continuous t (no FFT):
//   R = sum_band W_k e^{i phi_k},  phi_k = -Psi(f_k) + 2 pi f_k t,
//   rho^2 = |R|^2 P_tot / Q,  Q = P[k_hi] - P[k_lo]  (Eqs. 3-4; A cancels),
//   d rho^2/dt  = (P_tot/Q) 2 Re(conj R * 2 pi i sum W e^{i phi} f_k),
//   d rho^2/dm  = (P_tot/Q) 2 Re(conj R * (-2 pi i) sum W e^{i phi} dpsi_k/dm).
// The phase is FP64 at every bin (psi in turns, reduced mod 1), sincos and the
// products in FP32; per-thread FP32 partial sums, FP64 block and row totals in
// a fixed order (deterministic).  The time is split t = j dt + tau so that
// f_k t = (k j mod N)/N + k df tau with the first term exact in integers.
#include "mf_fft.cuh"
#include "mf_internal.h"
#include "mf_tmpl.cuh"

namespace mf {

constexpr int kRefThreads = 256;
constexpr int kRefBlocksPerRow = 16;
int refine_blocks_per_row() { return kRefBlocksPerRow; }

struct RefRow {
    double c[4];     // psi coefficients for u^1, u^2, u^3, u^5 (turns)
    float d1[4], d2[4];  // dpsi/dm1, dpsi/dm2 coefficients (turns per Msun)
    double dftau;    // df * tau (turns per bin)
    double pratio;   // P_tot / Q
    int64_t k_lo, k_hi;
    uint32_t j;      // nearest sample (mod N)
};

__device__ void refine_row_setup(const SegDev &seg, double f_low, const double *theta, const int64_t *band,
                                 int64_t i, RefRow &r) {
    const double m1 = theta[3 * i], m2 = theta[3 * i + 1], t = theta[3 * i + 2];
    double rec[kTmplStride];
    template_constants(m1, m2, rec);
    r.c[0] = rec[TF_C1]; r.c[1] = rec[TF_C2]; r.c[2] = rec[TF_C3]; r.c[3] = rec[TF_C5];
    double d1[4], d2[4];
    template_mass_derivs(m1, m2, d1, d2);
    for (int q = 0; q < 4; ++q) { r.d1[q] = (float)d1[q]; r.d2[q] = (float)d2[q]; }
    int64_t lo, hi;
    if (band) {
        lo = band[2 * i];
        hi = band[2 * i + 1];
    } else {
        const double N = (double)seg.N, fs = seg.fs;
        const double fisco = rec[TF_FISCO];
        const double fc = fisco < 0.5 * fs ? fisco : 0.5 * fs;
        lo = (int64_t)ceil(f_low * N / fs);
        hi = (int64_t)floor(fc * N / fs) + 1;
    }
    if (lo < 1) lo = 1;
    if (hi > seg.N / 2) hi = seg.N / 2;
    if (hi < lo) hi = lo;
    r.k_lo = lo;
    r.k_hi = hi;
    const double Q = seg.P[hi] - seg.P[lo];
    r.pratio = Q > 0.0 ? seg.consts->P_tot / Q : 0.0;
    const double x = t * seg.fs;
    const double jn = floor(x + 0.5);
    const double tau = (x - jn) / seg.fs;
    int64_t j = (int64_t)jn % seg.N;
    if (j < 0) j += seg.N;
    r.j = (uint32_t)j;
    r.dftau = seg.df * tau;
}

__global__ void __launch_bounds__(kRefThreads)
    k_refine_partial(SegDev seg, double f_low, const double *__restrict__ theta, const int64_t *__restrict__ band,
                     double *__restrict__ partial) {
    __shared__ RefRow row;
    __shared__ double red[8][kRefThreads / 32];
    const int64_t i = blockIdx.y;
    if (threadIdx.x == 0) refine_row_setup(seg, f_low, theta, band, i, row);
    __syncthreads();
    const int64_t K = row.k_hi - row.k_lo;
    const int64_t chunk = (K + gridDim.x - 1) / gridDim.x;
    const int64_t k0 = row.k_lo + (int64_t)blockIdx.x * chunk;
    const int64_t k1 = (k0 + chunk < row.k_hi) ? k0 + chunk : row.k_hi;
    const uint32_t nmask = (uint32_t)(seg.N - 1);
    const double invN = 1.0 / (double)seg.N;
    float ar = 0.f, ai = 0.f, fr = 0.f, fi = 0.f, ar1 = 0.f, ai1 = 0.f, ar2 = 0.f, ai2 = 0.f;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const double f = (double)k * seg.df;
        // u = f^(-1/3): FP32 seed refined by one FP64 Newton step
        double u = (double)rcbrtf((float)f);
        u = u * (4.0 - f * u * u * u) / 3.0;
        const double psi = -0.125 + u * (row.c[0] + u * (row.c[1] + u * (row.c[2] + u * u * row.c[3])));
        const double tt = (double)(((uint32_t)k * row.j) & nmask) * invN + (double)k * row.dftau;
        double ph = tt - psi;
        ph -= rint(ph);
        float s, c;
        __sincosf(6.283185307179586f * (float)ph, &s, &c);
        const float2 w = __ldg(&seg.W[k]);
        const float qr = w.x * c - w.y * s, qi = w.x * s + w.y * c;
        const float uf = (float)u, uf2 = uf * uf, uf3 = uf2 * uf, uf5 = uf3 * uf2;
        const float g1 = row.d1[0] * uf + row.d1[1] * uf2 + row.d1[2] * uf3 + row.d1[3] * uf5;
        const float g2 = row.d2[0] * uf + row.d2[1] * uf2 + row.d2[2] * uf3 + row.d2[3] * uf5;
        const float ff = (float)f;
        ar += qr; ai += qi;
        fr = fmaf(qr, ff, fr); fi = fmaf(qi, ff, fi);
        ar1 = fmaf(qr, g1, ar1); ai1 = fmaf(qi, g1, ai1);
        ar2 = fmaf(qr, g2, ar2); ai2 = fmaf(qi, g2, ai2);
    }
    double v[8] = {ar, ai, fr, fi, ar1, ai1, ar2, ai2};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        if (lane == 0) red[q][warp] = v[q];
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        double s = 0.0;
        for (int w = 0; w < kRefThreads / 32; ++w) s += red[threadIdx.x][w];
        partial[(i * gridDim.x + blockIdx.x) * 8 + threadIdx.x] = s;
    }
}

__global__ void k_refine_final(SegDev seg, double f_low, const double *__restrict__ theta,
                               const int64_t *__restrict__ band, const double *__restrict__ partial, int bpr,
                               int64_t n, double *__restrict__ obj, double *__restrict__ grad) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    RefRow row;
    refine_row_setup(seg, f_low, theta, band, i, row);
    double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < bpr; ++b)
        for (int q = 0; q < 8; ++q) a[q] += partial[(i * bpr + b) * 8 + q];
    const double Rr = a[0], Ri = a[1];
    const double pr = row.pratio;
    obj[i] = (Rr * Rr + Ri * Ri) * pr;
    const double two_pi = 2.0 * kPiD;
    // 2 Re(conj(R) * (i X)) = 2 (Ri Xr - Rr Xi)
    grad[3 * i + 0] = -two_pi * pr * 2.0 * (Ri * a[4] - Rr * a[5]);
    grad[3 * i + 1] = -two_pi * pr * 2.0 * (Ri * a[6] - Rr * a[7]);
    grad[3 * i + 2] = two_pi * pr * 2.0 * (Ri * a[2] - Rr * a[3]);
}

cudaError_t launch_refine(const SegDev &seg, double f_low, int phase_mode, const double *theta, int64_t n,
                          const int64_t *band, double *obj, double *grad, double *partial, cudaStream_t st) {
    (void)phase_mode;
    k_refine_partial<<<dim3(kRefBlocksPerRow, (unsigned)n), kRefThreads, 0, st>>>(seg, f_low, theta, band, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_refine_final<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(seg, f_low, theta, band, partial,
                                                                 kRefBlocksPerRow, n, obj, grad);
    return cudaGetLastError();
}

cudaError_t refine_kernel_attributes() { return cudaSuccess; }

}  // namespace mf
