// mf_refine.cu -- objective and adjoint for gradient refinement of triggers.
// For theta = (m1, m2, t) and a fixed band [k_lo, k_hi), Eq. (1) evaluated
// directly at continuous t (no FFT):
//   R = sum_band W_k e^{i phi_k},  phi_k = -Psi(f_k) + 2 pi f_k t,
//   rho^2 = |R|^2 P_tot / Q,  Q = P[k_hi] - P[k_lo]  (Eqs. 3-4; A cancels),
//   d rho^2/dt  = (P_tot/Q) 2 Re(conj R * 2 pi i sum W e^{i phi} f_k),
//   d rho^2/dm  = (P_tot/Q) 2 Re(conj R * (-2 pi i) sum W e^{i phi} dpsi_k/dm).
// The time is split t = j dt + tau so that f_k t = (k j mod N)/N + k df tau,
// the first term exact in integers and the second below a quarter turn.
// Phase forms (the bank's phase_mode):
//   anchors (default, also for the FP32-only mode): psi in FP64 at the centre
//     of every D = 2^log2D bins, reduced mod 1, with its first four
//     derivatives; FP32 quartic Taylor between anchors (the filter's form; D
//     from the same remainder bound, per row);
//   FP64 per bin: psi in FP64 at every bin, reduced mod 1.
// sincos and the products in FP32; per-thread FP32 partial sums, FP64 block
// and row totals in a fixed order (deterministic for a given blocks-per-row).
#include "mf_filter.cuh"
#include "mf_tmpl.cuh"

namespace mf {

constexpr int kRefThreads = 256;
constexpr int kRefBlocksPerRow = 16;          // the allocation-free entry point's (fixed scratch layout)
constexpr int kRefMinBlocksPerRow = 2;
constexpr int kRefMaxBlocksPerRow = 256;
constexpr int kRefAnchorsPerChunk = kRefThreads;
constexpr int64_t kRefMaxGridRows = 65535;    // rows per launch of the partial-sum kernel (grid y)
int refine_blocks_per_row() { return kRefBlocksPerRow; }

// The segments of one call, passed by value as a kernel parameter: row i
// reads segment row_seg[i] (0 when row_seg is NULL).
template <int NS>
struct SegTable {
    SegDev s[NS];
    int n;
};

int refine_blocks_for(int64_t n, int n_sm) {
    // about six blocks per SM over the whole call: each block pays a fixed
    // cost (its anchors in FP64, barriers, the 8-sum reduction), so more blocks
    // per row only help until the GPU is full (measured on 256 rows: 4 blocks
    // per row 2.4 ms, 16 per row 4.1 ms)
    int64_t b = (6 * (int64_t)n_sm + n - 1) / (n > 0 ? n : 1);
    if (b < kRefMinBlocksPerRow) b = kRefMinBlocksPerRow;
    if (b > kRefMaxBlocksPerRow) b = kRefMaxBlocksPerRow;
    return (int)b;
}

struct RefRow {
    double c[4];     // psi coefficients for u^1, u^2, u^3, u^5 (turns)
    float d1[4], d2[4];  // dpsi/dm1, dpsi/dm2 coefficients (turns per Msun)
    double dftau;    // df * tau (turns per bin)
    double pratio;   // P_tot / Q
    int64_t k_lo, k_hi;
    uint32_t j;      // nearest sample (mod N)
    int log2D;       // anchor spacing (0: FP64 phase at every bin)
};

__device__ void refine_row_setup(const SegDev &seg, double f_low, int anchored, const double *theta,
                                 const int64_t *band, int64_t i, RefRow &r) {
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
    // clamp into [1, N/2]: P has N/2 + 1 entries, so both edges stay readable
    // whatever band the caller passes (an edge beyond N/2 gives an empty band)
    const int64_t kmax = seg.N / 2;
    if (lo < 1) lo = 1;
    if (lo > kmax) lo = kmax;
    if (hi > kmax) hi = kmax;
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
    r.log2D = 0;
    if (anchored) {
        const double f0 = (double)lo * seg.df;
        r.log2D = anchor_log2D(psi_deriv_bound_u(r.c, f0, 1), psi_deriv_bound_u(r.c, f0, 5), seg.df);
    }
}

static_assert(sizeof(RefRow) <= kRefRowBytesMax, "row record larger than the scratch layout allows");

size_t refine_scratch_bytes(int64_t n, int bpr) {
    return sizeof(double) * 8 * (size_t)bpr * (size_t)n + kRefRowBytesMax * (size_t)n;
}

// the row records follow the per-block partial sums in the scratch
__device__ __host__ __forceinline__ RefRow *row_records(double *partial, int bpr, int64_t n) {
    return reinterpret_cast<RefRow *>(partial + 8 * (size_t)bpr * (size_t)n);
}

// The mass-derivative weights g_m(k) = dpsi/dm(f_k) = sum_p d_p u^p at an
// anchor centre k_a, with their first two k-derivatives (u = (k df)^(-1/3),
// du/dk = -u/(3k), d2u/dk2 = 4u/(9k^2)): g(k_a + d) ~ g + g' d + g'' d^2 / 2
// within the anchor's D <= 256 bins (relative error ~ (D/2k)^3 < 2e-6 at f_low).
__device__ __forceinline__ void mass_weight_taylor(const float *dc, float u, float ik, float &g0, float &g1,
                                                   float &g2) {
    const float u2 = u * u, u3 = u2 * u, u4 = u2 * u2, u5 = u4 * u;
    const float g = dc[0] * u + dc[1] * u2 + dc[2] * u3 + dc[3] * u5;
    const float gu = dc[0] + 2.f * dc[1] * u + 3.f * dc[2] * u2 + 5.f * dc[3] * u4;
    const float guu = 2.f * dc[1] + 6.f * dc[2] * u + 20.f * dc[3] * u3;
    const float du = -u * ik * (1.f / 3.f), d2u = u * ik * ik * (4.f / 9.f);
    g0 = g;
    g1 = gu * du;
    g2 = 0.5f * (guu * du * du + gu * d2u);
}

struct RefAcc {
    float ar = 0.f, ai = 0.f, fr = 0.f, fi = 0.f, ar1 = 0.f, ai1 = 0.f, ar2 = 0.f, ai2 = 0.f;
    // one bin: phase (turns, reduced to [-1/2, 1/2]), the frequency and the
    // mass-derivative weights g1 = dpsi/dm1, g2 = dpsi/dm2 at the bin
    __device__ __forceinline__ void add_w(const float2 w, float ph, float ff, float g1, float g2) {
        float s, c;
        __sincosf(6.283185307179586f * ph, &s, &c);
        const float qr = w.x * c - w.y * s, qi = w.x * s + w.y * c;
        ar += qr; ai += qi;
        fr = fmaf(qr, ff, fr); fi = fmaf(qi, ff, fi);
        ar1 = fmaf(qr, g1, ar1); ai1 = fmaf(qi, g1, ai1);
        ar2 = fmaf(qr, g2, ar2); ai2 = fmaf(qi, g2, ai2);
    }
    __device__ __forceinline__ void add(const RefRow &row, const float2 w, float ph, float ff, float uf) {
        float s, c;
        __sincosf(6.283185307179586f * ph, &s, &c);
        const float qr = w.x * c - w.y * s, qi = w.x * s + w.y * c;
        const float uf2 = uf * uf, uf3 = uf2 * uf, uf5 = uf3 * uf2;
        const float g1 = row.d1[0] * uf + row.d1[1] * uf2 + row.d1[2] * uf3 + row.d1[3] * uf5;
        const float g2 = row.d2[0] * uf + row.d2[1] * uf2 + row.d2[2] * uf3 + row.d2[3] * uf5;
        ar += qr; ai += qi;
        fr = fmaf(qr, ff, fr); fi = fmaf(qi, ff, fi);
        ar1 = fmaf(qr, g1, ar1); ai1 = fmaf(qi, g1, ai1);
        ar2 = fmaf(qr, g2, ar2); ai2 = fmaf(qi, g2, ai2);
    }
};

// segment of row i, or -1 when row_seg names no segment of the table
template <int NS>
__device__ __forceinline__ int row_segment(const SegTable<NS> &tab, const int32_t *row_seg, int64_t i) {
    const int s = row_seg ? row_seg[i] : 0;
    return (s >= 0 && s < tab.n) ? s : -1;
}

// One thread per row: template constants, mass derivatives, band, time split
// and anchor spacing (FP64), once per row instead of once per block.
template <int NS>
__global__ void k_refine_setup(const __grid_constant__ SegTable<NS> tab, const int32_t *__restrict__ row_seg,
                               double f_low, int anchored, const double *__restrict__ theta,
                               const int64_t *__restrict__ band, int64_t n, RefRow *__restrict__ rows) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int si = row_segment(tab, row_seg, i);
    if (si < 0) return;   // the other kernels check the segment index themselves
    refine_row_setup(tab.s[si], f_low, anchored, theta, band, i, rows[i]);
}

template <int NS>
__global__ void __launch_bounds__(kRefThreads)
    k_refine_partial(const __grid_constant__ SegTable<NS> tab, const int32_t *__restrict__ row_seg,
                     const RefRow *__restrict__ rows, double *__restrict__ partial, int64_t i0) {
    __shared__ RefRow row;
    __shared__ double red[8][kRefThreads / 32];
    __shared__ float4 sanc[kRefAnchorsPerChunk];
    __shared__ float sanc4[kRefAnchorsPerChunk];
    __shared__ float4 sg[kRefAnchorsPerChunk];    // g1 Taylor (3), g2 value
    __shared__ float2 sg2[kRefAnchorsPerChunk];   // g2 first and second k-derivative terms
    const int64_t i = i0 + blockIdx.y;   // rows go in chunks of at most 65535 (grid y limit)
    const int si = row_segment(tab, row_seg, i);
    if (si < 0) {   // invalid segment index: an empty sum (the final kernel reports NaN)
        if (threadIdx.x < 8) partial[(i * gridDim.x + blockIdx.x) * 8 + threadIdx.x] = 0.0;
        return;
    }
    const SegDev &seg = tab.s[si];
    if (threadIdx.x == 0) row = rows[i];
    __syncthreads();
    const uint32_t nmask = (uint32_t)(seg.N - 1);
    RefAcc acc;
    if (row.log2D > 0) {
        // this block's anchor groups g (bins [g D, g D + D) clipped to the band)
        const int lg = row.log2D;
        const int64_t g_lo = row.k_lo >> lg, g_hi = (row.k_hi - 1) >> lg;
        const int64_t ng = row.k_hi > row.k_lo ? g_hi - g_lo + 1 : 0;
        const int64_t gpb = (ng + gridDim.x - 1) / gridDim.x;
        const int64_t gb0 = g_lo + (int64_t)blockIdx.x * gpb;
        const int64_t gb1 = (gb0 + gpb < g_lo + ng) ? gb0 + gpb : g_lo + ng;
        const float invN = 1.0f / (float)seg.N;
        const float dftau = (float)row.dftau, dff = (float)seg.df;
        const int half = (1 << lg) >> 1;
        for (int64_t gc = gb0; gc < gb1; gc += kRefAnchorsPerChunk) {
            const int64_t gce = (gc + kRefAnchorsPerChunk < gb1) ? gc + kRefAnchorsPerChunk : gb1;
            if (gc + threadIdx.x < gce) {
                const int64_t g = gc + threadIdx.x;
                anchor_record(row.c[0], row.c[1], row.c[2], row.c[3], g, lg, seg.df, sanc[threadIdx.x],
                              sanc4[threadIdx.x]);
                const float ka = (float)((g << lg) + half);
                const float u = rcbrtf(ka * (float)seg.df), ik = 1.f / ka;
                float a0, a1, a2, b0, b1, b2;
                mass_weight_taylor(row.d1, u, ik, a0, a1, a2);
                mass_weight_taylor(row.d2, u, ik, b0, b1, b2);
                sg[threadIdx.x] = make_float4(a0, a1, a2, b0);
                sg2[threadIdx.x] = make_float2(b1, b2);
            }
            __syncthreads();
            int64_t kb0 = gc << lg, kb1 = gce << lg;
            if (kb0 < row.k_lo) kb0 = row.k_lo;
            if (kb1 > row.k_hi) kb1 = row.k_hi;
            for (int64_t k = kb0 + threadIdx.x; k < kb1; k += kRefThreads) {
                const int a = (int)((k >> lg) - gc);
                const float4 an = sanc[a];
                const float d = (float)(int)((k & ((1 << lg) - 1)) - half);
                const float psi = an.x + d * (an.y + d * (an.z + d * (an.w + d * sanc4[a])));
                const float tt = (float)(((uint32_t)k * row.j) & nmask) * invN + (float)k * dftau;
                float ph = tt - psi;
                ph -= rintf(ph);
                const float ff = (float)k * dff;
                const float4 ga = sg[a];
                const float2 gb = sg2[a];
                const float g1 = fmaf(fmaf(ga.z, d, ga.y), d, ga.x);
                const float g2 = fmaf(fmaf(gb.y, d, gb.x), d, ga.w);
                acc.add_w(__ldg(&seg.W[k]), ph, ff, g1, g2);
            }
            __syncthreads();
        }
    } else {
        const int64_t K = row.k_hi - row.k_lo;
        const int64_t chunk = (K + gridDim.x - 1) / gridDim.x;
        const int64_t k0 = row.k_lo + (int64_t)blockIdx.x * chunk;
        const int64_t k1 = (k0 + chunk < row.k_hi) ? k0 + chunk : row.k_hi;
        const double invN = 1.0 / (double)seg.N;
        for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            const double f = (double)k * seg.df;
            // u = f^(-1/3): FP32 seed refined by one FP64 Newton step
            double u = (double)rcbrtf((float)f);
            u = u * (4.0 - f * u * u * u) * (1.0 / 3.0);
            const double psi = -0.125 + u * (row.c[0] + u * (row.c[1] + u * (row.c[2] + u * u * row.c[3])));
            const double tt = (double)(((uint32_t)k * row.j) & nmask) * invN + (double)k * row.dftau;
            double ph = tt - psi;
            ph -= rint(ph);
            acc.add(row, __ldg(&seg.W[k]), (float)ph, (float)f, (float)u);
        }
    }
    double v[8] = {acc.ar, acc.ai, acc.fr, acc.fi, acc.ar1, acc.ai1, acc.ar2, acc.ai2};
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

template <int NS>
__global__ void k_refine_final(const __grid_constant__ SegTable<NS> tab, const int32_t *__restrict__ row_seg,
                               const RefRow *__restrict__ rows, const double *__restrict__ partial, int bpr,
                               int64_t n, double *__restrict__ obj, double *__restrict__ grad) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int si = row_segment(tab, row_seg, i);
    if (si < 0) {
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        obj[i] = nan;
        grad[3 * i] = grad[3 * i + 1] = grad[3 * i + 2] = nan;
        return;
    }
    double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < bpr; ++b)
        for (int q = 0; q < 8; ++q) a[q] += partial[(i * bpr + b) * 8 + q];
    const double Rr = a[0], Ri = a[1];
    const double pr = rows[i].pratio;
    obj[i] = (Rr * Rr + Ri * Ri) * pr;
    const double two_pi = 2.0 * kPiD;
    // 2 Re(conj(R) * (i X)) = 2 (Ri Xr - Rr Xi)
    grad[3 * i + 0] = -two_pi * pr * 2.0 * (Ri * a[4] - Rr * a[5]);
    grad[3 * i + 1] = -two_pi * pr * 2.0 * (Ri * a[6] - Rr * a[7]);
    grad[3 * i + 2] = two_pi * pr * 2.0 * (Ri * a[2] - Rr * a[3]);
}

template <int NS>
static cudaError_t launch_refine_table(const SegTable<NS> &tab, const int32_t *row_seg, double f_low,
                                       int phase_mode, const double *theta, int64_t n, const int64_t *band,
                                       double *obj, double *grad, double *partial, int bpr, cudaStream_t st) {
    const int anchored = phase_mode == MF_PHASE_FP64 ? 0 : 1;
    RefRow *rows = row_records(partial, bpr, n);
    k_refine_setup<NS><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(tab, row_seg, f_low, anchored, theta, band, n,
                                                                     rows);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int64_t i0 = 0; i0 < n; i0 += kRefMaxGridRows) {
        const int64_t rows_here = n - i0 < kRefMaxGridRows ? n - i0 : kRefMaxGridRows;
        k_refine_partial<NS><<<dim3((unsigned)bpr, (unsigned)rows_here), kRefThreads, 0, st>>>(tab, row_seg, rows,
                                                                                              partial, i0);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_refine_final<NS><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(tab, row_seg, rows, partial, bpr, n, obj, grad);
    return cudaGetLastError();
}

cudaError_t launch_refine(const SegDev &seg, double f_low, int phase_mode, const double *theta, int64_t n,
                          const int64_t *band, double *obj, double *grad, double *partial, int bpr,
                          cudaStream_t st) {
    SegTable<1> tab;
    tab.s[0] = seg;
    tab.n = 1;
    return launch_refine_table(tab, nullptr, f_low, phase_mode, theta, n, band, obj, grad, partial, bpr, st);
}

cudaError_t launch_refine_multi(const SegDev *segs, int n_seg, const int32_t *row_seg, double f_low,
                                int phase_mode, const double *theta, int64_t n, const int64_t *band, double *obj,
                                double *grad, double *partial, int bpr, cudaStream_t st) {
    if (n_seg < 1 || n_seg > kRefineMaxSegs) return cudaErrorInvalidValue;
    if (n_seg <= 8) {
        SegTable<8> tab;
        for (int s = 0; s < n_seg; ++s) tab.s[s] = segs[s];
        tab.n = n_seg;
        return launch_refine_table(tab, row_seg, f_low, phase_mode, theta, n, band, obj, grad, partial, bpr, st);
    }
    SegTable<kRefineMaxSegs> tab;
    for (int s = 0; s < n_seg; ++s) tab.s[s] = segs[s];
    tab.n = n_seg;
    return launch_refine_table(tab, row_seg, f_low, phase_mode, theta, n, band, obj, grad, partial, bpr, st);
}

cudaError_t refine_kernel_attributes() { return cudaSuccess; }

}  // namespace mf
