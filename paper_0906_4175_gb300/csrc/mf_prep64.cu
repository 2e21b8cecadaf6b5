// mf_prep64.cu -- the forward DFT of segment conditioning in FP64:
//   X_k = sum_n s_n e^{-2 pi i n k / N},  k = 0 .. N/2  (rounded to complex64)
// for the weighting W_k = a_k conj(X_k) of Eq. (1).
//
// Why FP64: detector data carry far more power below f_low than inside the
// band (the f^-56 wall of Eq. 2), and an FP32 FFT spreads round-off of the
// order of the largest components' size over every output bin.  In FP64 that
// round-off stays ~1e-16 of the total, so the in-band bins keep their FP32
// precision whatever the out-of-band content; only the final rounding of each
// bin to complex64 remains, relative to that bin's own size.
//
// Real input of N samples as one complex DFT of M = N/2 points,
// z_n = s_{2n} + i s_{2n+1}:  with Z = DFT_M(z),
//   X_k = (Z_k + conj Z_{M-k}) / 2 + e^{-2 pi i k/N} (Z_k - conj Z_{M-k}) / (2i),
// the even / odd-sample split of the DFT.  DFT_M is a four-step transform
// M = M1 M2 (M2 = 2^floor(log2 M / 2) columns of stride M1):
//   pass A  column DFTs of length M2 (one CTA per group of columns, radix-4
//           Stockham stages in shared memory), times e^{-2 pi i n1 k2 / M},
//           written transposed, E[k2 M1 + n1];
//   pass B  row DFTs of length M1 in place (Z_{k2 + M2 k1} = E'[k2 M1 + k1]);
//   split   X_k from Z_k and Z_{M-k}.
// Twiddles: exp(-2 pi i m / P) for P = 2^p as hi[m >> 10] * lo[m & 1023]
// (FP64 sincospi of exact arguments, once per device).
#include <algorithm>

#include "mf_internal.h"

namespace mf {
namespace {

constexpr int kRootLo = 1024;
// table layout per p = 4 .. 22: lo (min(P, 1024) entries) then hi (max(1, P/1024))
__host__ __device__ constexpr int root_lo_size(int p) { return p >= 10 ? kRootLo : (1 << p); }
__host__ __device__ constexpr int root_hi_size(int p) { return p >= 10 ? (1 << (p - 10)) : 1; }
// closed form of the running sum of (lo + hi) over p' = 4 .. p-1
__host__ __device__ constexpr int root_offset(int p) {
    return p <= 10 ? ((1 << p) - 16) + (p - 4) : 1014 + kRootLo * (p - 10) + ((1 << (p - 10)) - 1);
}
constexpr int kRootTotal = root_offset(23);
static_assert(root_offset(11) == root_offset(10) + kRootLo + 1 && root_offset(5) == 17, "table layout");
static __device__ double2 g_roots64[kRootTotal];

__global__ void k_init_roots64() {
    for (int p = 4; p <= 22; ++p) {
        double2 *lo = g_roots64 + root_offset(p);
        double2 *hi = lo + root_lo_size(p);
        const double P = (double)(1ll << p);
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < root_lo_size(p); j += gridDim.x * blockDim.x) {
            double sn, cs;
            sincospi(-2.0 * (double)j / P, &sn, &cs);
            lo[j] = make_double2(cs, sn);
        }
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < root_hi_size(p); i += gridDim.x * blockDim.x) {
            double sn, cs;
            sincospi(-2.0 * (double)i * (double)kRootLo / P, &sn, &cs);
            hi[i] = make_double2(cs, sn);
        }
    }
}

__device__ __forceinline__ double2 dmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 dadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 dsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// exp(-2 pi i m / 2^p), 0 <= m < 2^p
__device__ __forceinline__ double2 root64(int64_t m, int p) {
    const double2 *lo = g_roots64 + root_offset(p);
    if (p <= 10) return __ldg(&lo[m]);
    const double2 *hi = lo + kRootLo;
    return dmul(__ldg(&hi[m >> 10]), __ldg(&lo[m & (kRootLo - 1)]));
}

// In-place forward DFT (sign -1) of S sequences of length L = 2^LG held in
// shared memory (sequence q at x + q L), natural order in and out, by all NT
// threads of the CTA: radix-4 Stockham stages, then one radix-2 stage when LG
// is odd.  Each stage loads all of a thread's butterflies, synchronises, and
// writes them back.
template <int LG, int S, int NT>
__device__ __forceinline__ void smem_dft64(double2 *x) {
    constexpr int L = 1 << LG;
    constexpr int B4 = S * L / 4;               // radix-4 butterflies per stage
    constexpr int PT = (B4 + NT - 1) / NT;      // per thread
#pragma unroll
    for (int st = 0; st + 2 <= LG; st += 2) {
        const int lgNs = st, Ns = 1 << st;   // size of the sub-transforms done so far
        double2 v[PT][4];
#pragma unroll
        for (int i = 0; i < PT; ++i) {
            const int bb = threadIdx.x + i * NT;
            if (bb < B4) {
                const int q = bb >> (LG - 2), b = bb & (L / 4 - 1);
                const double2 *xs = x + q * L;
#pragma unroll
                for (int r = 0; r < 4; ++r) v[i][r] = xs[b + r * (L / 4)];
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < PT; ++i) {
            const int bb = threadIdx.x + i * NT;
            if (bb < B4) {
                const int q = bb >> (LG - 2), b = bb & (L / 4 - 1);
                const int j = b & (Ns - 1), g = b >> lgNs;
                double2 x0 = v[i][0], x1 = v[i][1], x2 = v[i][2], x3 = v[i][3];
                if (Ns > 1) {   // exp(-2 pi i j r / (4 Ns)) on input r
                    x1 = dmul(x1, root64(j, lgNs + 2));
                    x2 = dmul(x2, root64(2 * j, lgNs + 2));
                    x3 = dmul(x3, root64(3 * j, lgNs + 2));
                }
                const double2 a = dadd(x0, x2), c = dsub(x0, x2);
                const double2 e = dadd(x1, x3), d = dsub(x1, x3);
                double2 *ys = x + q * L + g * 4 * Ns + j;
                ys[0] = dadd(a, e);
                ys[Ns] = make_double2(c.x + d.y, c.y - d.x);        // c - i d
                ys[2 * Ns] = dsub(a, e);
                ys[3 * Ns] = make_double2(c.x - d.y, c.y + d.x);    // c + i d
            }
        }
        __syncthreads();
    }
    if constexpr (LG % 2 == 1) {
        constexpr int B2 = S * L / 2;
        constexpr int PT2 = (B2 + NT - 1) / NT;
        double2 v[PT2][2];
#pragma unroll
        for (int i = 0; i < PT2; ++i) {
            const int bb = threadIdx.x + i * NT;
            if (bb < B2) {
                const int q = bb >> (LG - 1), b = bb & (L / 2 - 1);
                v[i][0] = x[q * L + b];
                v[i][1] = x[q * L + b + L / 2];
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < PT2; ++i) {
            const int bb = threadIdx.x + i * NT;
            if (bb < B2) {   // last stage: Ns = L/2, g = 0
                const int q = bb >> (LG - 1), j = bb & (L / 2 - 1);
                const double2 t = L > 2 ? dmul(v[i][1], root64(j, LG)) : v[i][1];
                x[q * L + j] = dadd(v[i][0], t);
                x[q * L + j + L / 2] = dsub(v[i][0], t);
            }
        }
        __syncthreads();
    }
}

constexpr int kNT = 256;

__host__ __device__ constexpr int cx_log2(int x) { return x <= 1 ? 0 : 1 + cx_log2(x >> 1); }

// sequences of length 2^LG per CTA: 1024 points in shared memory (16 KB;
// 2048 for the longest rows), one radix-4 butterfly per thread and stage
template <int LG>
__host__ __device__ constexpr int seqs64() { return LG >= 10 ? 1 : (1024 >> LG); }

// pass A: columns n1 of z (stride M1, M2 = 2^LG2 points each), ca = min(seqs64, M1) per CTA
template <int LG2>
__global__ void __launch_bounds__(kNT) k_fwd64_cols(const float2 *__restrict__ z, int lgM, double2 *__restrict__ E) {
    constexpr int L = 1 << LG2, S = seqs64<LG2>();
    extern __shared__ double2 sm64[];
    const int lgM1 = lgM - LG2;
    const int64_t M1 = (int64_t)1 << lgM1;
    const int lgca = lgM1 < cx_log2(S) ? lgM1 : cx_log2(S);
    const int ca = 1 << lgca;
    const int64_t n1_0 = (int64_t)blockIdx.x * ca;
    for (int e = threadIdx.x; e < ca * L; e += kNT) {   // consecutive threads: consecutive columns
        const int c = e & (ca - 1), n2 = e >> lgca;
        const float2 v = z[n1_0 + c + n2 * M1];
        sm64[c * L + n2] = make_double2((double)v.x, (double)v.y);
    }
    __syncthreads();
    smem_dft64<LG2, S, kNT>(sm64);   // sequences ca .. S-1 (if any) hold no data and are not stored
    for (int e = threadIdx.x; e < ca * L; e += kNT) {
        const int c = e & (ca - 1), k2 = e >> lgca;
        const int64_t n1 = n1_0 + c;
        E[(int64_t)k2 * M1 + n1] = dmul(sm64[c * L + k2], root64(n1 * k2, lgM));
    }
}

// pass B: rows k2 of E (M1 = 2^LG1 points each, contiguous), cb = min(seqs64, M2) per CTA, in place
template <int LG1>
__global__ void __launch_bounds__(kNT) k_fwd64_rows(double2 *__restrict__ E, int lgM) {
    constexpr int L = 1 << LG1, S = seqs64<LG1>();
    extern __shared__ double2 sm64[];
    const int64_t M2 = (int64_t)1 << (lgM - LG1);
    const int cb = M2 < S ? (int)M2 : S;
    double2 *row = E + (int64_t)blockIdx.x * cb * L;
    for (int e = threadIdx.x; e < cb * L; e += kNT) sm64[e] = row[e];
    __syncthreads();
    smem_dft64<LG1, S, kNT>(sm64);
    for (int e = threadIdx.x; e < cb * L; e += kNT) row[e] = sm64[e];
}

// X_k, k = 0 .. M, from Z (Z_k at E[(k mod M2) M1 + k div M2])
__global__ void k_fwd64_split(const double2 *__restrict__ Z, int lgM, float2 *__restrict__ X) {
    const int lgM2 = lgM / 2, lgM1 = lgM - lgM2;
    const int64_t M = (int64_t)1 << lgM;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= M; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ka = k & (M - 1), kb = (M - k) & (M - 1);
        const double2 za = Z[((ka & (((int64_t)1 << lgM2) - 1)) << lgM1) + (ka >> lgM2)];
        const double2 zb = Z[((kb & (((int64_t)1 << lgM2) - 1)) << lgM1) + (kb >> lgM2)];
        const double2 ev = make_double2(0.5 * (za.x + zb.x), 0.5 * (za.y - zb.y));   // (Z_k + conj Z_{M-k}) / 2
        const double2 od = make_double2(0.5 * (za.y + zb.y), -0.5 * (za.x - zb.x));  // (Z_k - conj Z_{M-k}) / (2i)
        const double2 x = dadd(ev, dmul(od, root64(k & ((M << 1) - 1), lgM + 1)));
        X[k] = make_float2((float)x.x, (float)x.y);
    }
}

template <int LG>
constexpr size_t smem64_bytes() { return (size_t)seqs64<LG>() * (1 << LG) * sizeof(double2); }

template <int LG2>
cudaError_t launch_cols(const float2 *z, int lgM, double2 *E, cudaStream_t st, bool attrs) {
    if (attrs)
        return cudaFuncSetAttribute(k_fwd64_cols<LG2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem64_bytes<LG2>());
    const int64_t M1 = (int64_t)1 << (lgM - LG2);
    const int64_t ca = std::min<int64_t>(M1, seqs64<LG2>());
    k_fwd64_cols<LG2><<<(unsigned)(M1 / ca), kNT, smem64_bytes<LG2>(), st>>>(z, lgM, E);
    return cudaGetLastError();
}
template <int LG1>
cudaError_t launch_rows(double2 *E, int lgM, cudaStream_t st, bool attrs) {
    if (attrs)
        return cudaFuncSetAttribute(k_fwd64_rows<LG1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem64_bytes<LG1>());
    const int64_t M2 = (int64_t)1 << (lgM - LG1);
    const int64_t cb = std::min<int64_t>(M2, seqs64<LG1>());
    k_fwd64_rows<LG1><<<(unsigned)(M2 / cb), kNT, smem64_bytes<LG1>(), st>>>(E, lgM);
    return cudaGetLastError();
}

// M = 2^lgM, lgM = 9 .. 21: column length 2^(lgM/2), row length 2^(lgM - lgM/2)
cudaError_t fwd64_passes(const float2 *z, int lgM, double2 *E, cudaStream_t st, bool attrs) {
    cudaError_t e = cudaSuccess;
    switch (lgM / 2) {
        case 4: e = launch_cols<4>(z, lgM, E, st, attrs); break;
        case 5: e = launch_cols<5>(z, lgM, E, st, attrs); break;
        case 6: e = launch_cols<6>(z, lgM, E, st, attrs); break;
        case 7: e = launch_cols<7>(z, lgM, E, st, attrs); break;
        case 8: e = launch_cols<8>(z, lgM, E, st, attrs); break;
        case 9: e = launch_cols<9>(z, lgM, E, st, attrs); break;
        case 10: e = launch_cols<10>(z, lgM, E, st, attrs); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    switch (lgM - lgM / 2) {
        case 5: return launch_rows<5>(E, lgM, st, attrs);
        case 6: return launch_rows<6>(E, lgM, st, attrs);
        case 7: return launch_rows<7>(E, lgM, st, attrs);
        case 8: return launch_rows<8>(E, lgM, st, attrs);
        case 9: return launch_rows<9>(E, lgM, st, attrs);
        case 10: return launch_rows<10>(E, lgM, st, attrs);
        case 11: return launch_rows<11>(E, lgM, st, attrs);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// s: N float32 samples (device, 8-byte aligned); scratch: N/2 complex128
// (8 N bytes); X: N/2 + 1 complex64.  Three kernels.
cudaError_t launch_forward_fft64(const float *s, int64_t N, void *scratch, float2 *X, cudaStream_t st) {
    int lgN = 0;
    while (((int64_t)1 << (lgN + 1)) <= N) ++lgN;
    const int lgM = lgN - 1;
    if (lgM < 9 || lgM > 21) return cudaErrorInvalidValue;
    double2 *E = (double2 *)scratch;
    cudaError_t e = fwd64_passes(reinterpret_cast<const float2 *>(s), lgM, E, st, false);
    if (e != cudaSuccess) return e;
    const int64_t M = N / 2;
    int blocks = (int)((M + 1 + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_fwd64_split<<<blocks, 256, 0, st>>>(E, lgM, X);
    return cudaGetLastError();
}

cudaError_t prep64_kernel_attributes() {
    k_init_roots64<<<32, 256>>>();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int lgM = 9; lgM <= 21; ++lgM)
        if ((e = fwd64_passes(nullptr, lgM, nullptr, nullptr, true)) != cudaSuccess) return e;
    return cudaDeviceSynchronize();
}

}  // namespace mf
