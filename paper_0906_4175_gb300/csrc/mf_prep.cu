// mf_prep.cu -- once-per-segment conditioning for Eq. (1) of arXiv:0906.4175:
//   X_k = DFT(s)_k (own four-step FP32 FFT, forward sign), k = 0..N/2
//   q_k = f_k^(-7/3) / S_k (FP32 powers of f and Eq. (2) bracket, FP64 result;
//         S_k = S0 [(4.49 x)^-56 + 0.16 x^-4.52 + 0.52 + 0.32 x^2], x = f/f0, or a caller table)
//   P_k = sum_{k' < k} q_k'  (FP64 exclusive prefix; sigma^2 of Eq. (4) for the
//         band [k_lo, k_hi) is 4 df A^2 (P[k_hi] - P[k_lo]))
//   W_k = alpha f_k^(-7/6) dt conj(X_k) / S_k, alpha = sqrt(4 df / P[N/2]),
// so that raw_j = sum_band W_k e^{-i Psi_k} e^{2 pi i j k/N} gives
// rho_j = |raw_j| sqrt(P[N/2] / (P[k_hi] - P[k_lo])) for any PSD scale.
#include "mf_passes.cuh"

namespace mf {

namespace {
struct FwdOp {
    const float *s;
    float2 *exch, *X;
    int log2N;
    cudaStream_t st;
    template <int N2, int N1>
    cudaError_t run() {
        constexpr int C1 = seqs_per_cta<N2>(N1);
        constexpr int C2 = seqs_per_cta<N1>(N2);
        const int log2N2 = log2_n2(log2N), log2N1 = log2N - log2N2;
        typename ColRealSrc<N2, C1, cx_ilog2(N1)>::Params sp{s, log2N1};
        typename ExchSink<N2, C1, -1, cx_ilog2(N1)>::Params kp{exch, log2N1, log2N};
        cudaError_t e = run_pass<N2, C1, true, -1, ColRealSrc<N2, C1, cx_ilog2(N1)>, ExchSink<N2, C1, -1, cx_ilog2(N1)>>(
            dim3(N1 / C1, 1), sp, kp, st);
        if (e != cudaSuccess) return e;
        typename RowSrc<N1, C2>::Params sp2{exch, log2N1, log2N};
        typename RowComplexOut<N1, C2>::Params kp2{X, log2N2, ((int64_t)1 << (log2N - 1)) + 1};
        return run_pass<N1, C2, false, -1, RowSrc<N1, C2>, RowComplexOut<N1, C2>>(dim3(N2 / C2, 1), sp2, kp2,
                                                                                  st);
    }
};
struct FwdAttrOp {
    template <int N2, int N1>
    cudaError_t run() {
        constexpr int C1 = seqs_per_cta<N2>(N1);
        constexpr int C2 = seqs_per_cta<N1>(N2);
        cudaError_t e = set_pass_attrs<N2, C1, true, -1, ColRealSrc<N2, C1, cx_ilog2(N1)>, ExchSink<N2, C1, -1, cx_ilog2(N1)>>();
        if (e != cudaSuccess) return e;
        return set_pass_attrs<N1, C2, false, -1, RowSrc<N1, C2>, RowComplexOut<N1, C2>>();
    }
};
}  // namespace

// Batched complex FFT y_b = sum_n x_b[n] e^{SIGN 2 pi i n k / N} (unnormalised),
// batch entries N apart, through the same four-step passes.
template <int SIGN>
struct C2COp {
    const float2 *x;
    float2 *y, *exch;
    int batch;
    cudaStream_t st;
    template <int N2, int N1>
    cudaError_t run() {
        constexpr int C1 = seqs_per_cta<N2>(N1);
        constexpr int C2 = seqs_per_cta<N1>(N2);
        constexpr int LG1 = cx_ilog2(N1), LG2 = cx_ilog2(N2);
        const int64_t N = (int64_t)N1 * N2;
        typename ColComplexSrc<N2, C1, false, LG1>::Params sp{x, LG1, N};
        typename ExchSink<N2, C1, SIGN, LG1>::Params kp{exch, LG1, LG1 + LG2};
        cudaError_t e = run_pass<N2, C1, true, SIGN, ColComplexSrc<N2, C1, false, LG1>, ExchSink<N2, C1, SIGN, LG1>>(
            dim3(N1 / C1, batch), sp, kp, st);
        if (e != cudaSuccess) return e;
        typename RowSrc<N1, C2>::Params sp2{exch, LG1, LG1 + LG2};
        typename RowTileOut<N1, C2>::Params kp2{y, LG2, N};
        return run_pass<N1, C2, false, SIGN, RowSrc<N1, C2>, RowTileOut<N1, C2>>(dim3(N2 / C2, batch), sp2, kp2, st);
    }
};
template <int SIGN>
struct C2CAttrOp {
    template <int N2, int N1>
    cudaError_t run() {
        constexpr int C1 = seqs_per_cta<N2>(N1);
        constexpr int C2 = seqs_per_cta<N1>(N2);
        constexpr int LG1 = cx_ilog2(N1);
        cudaError_t e = set_pass_attrs<N2, C1, true, SIGN, ColComplexSrc<N2, C1, false, LG1>, ExchSink<N2, C1, SIGN, LG1>>();
        if (e != cudaSuccess) return e;
        return set_pass_attrs<N1, C2, false, SIGN, RowSrc<N1, C2>, RowTileOut<N1, C2>>();
    }
};

// Single-pass batched FFT for N = L <= 2048: a CTA holds C = 8192/L whole
// sequences (one or two warps each) in shared memory, so every point is read
// and written once instead of twice through the four-step exchange.
// Sequence s of the batch is x[s L .. s L + L); CTAs past the batch load zeros
// and store nothing.
template <int L, int C>
struct SeqSrc {
    static constexpr bool kHalfZero = false;
    static constexpr size_t kScratchBytes = 0;
    struct Params { const float2 *x; int64_t n_seq; };
    const Params &p;
    const int tile;
    __device__ SeqSrc(const Params &pp, int tl, int, int, void *) : p(pp), tile(tl) {}
    __device__ __forceinline__ void load(int seq, int t, float2 *v) const {
        constexpr int T = L / 32;
        const int64_t s = (int64_t)tile * C + seq;
        if (s >= p.n_seq) {
#pragma unroll
            for (int r = 0; r < 32; ++r) v[r] = czero();
            return;
        }
        const float2 *x = p.x + s * L;
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = __ldcs(&x[t + r * T]);
    }
};
template <int L, int C>
struct SeqOut {
    struct Params { float2 *y; int64_t n_seq; };
    const Params &p;
    const int tile;
    __device__ SeqOut(const Params &pp, int tl, int, int) : p(pp), tile(tl) {}
    template <int R>
    __device__ __forceinline__ void store(int seq, int b, int stride, const float2 *v) const {
        const int64_t s = (int64_t)tile * C + seq;
        if (s >= p.n_seq) return;
        float2 *y = p.y + s * L;
#pragma unroll
        for (int r = 0; r < R; ++r) __stcs(&y[b + r * stride], v[r]);
    }
    __device__ __forceinline__ void finish(float2 *) const {}
};

template <int L, int SIGN>
static cudaError_t run_c2c_single(const float2 *x, float2 *y, int64_t batch, cudaStream_t st) {
    constexpr int C = 8192 / L;
    typename SeqSrc<L, C>::Params sp{x, batch};
    typename SeqOut<L, C>::Params kp{y, batch};
    return run_pass<L, C, false, SIGN, SeqSrc<L, C>, SeqOut<L, C>>(dim3((unsigned)((batch + C - 1) / C), 1), sp,
                                                                   kp, st);
}

template <int SIGN>
static cudaError_t c2c_single_attrs() {
    cudaError_t e = set_pass_attrs<1024, 8, false, SIGN, SeqSrc<1024, 8>, SeqOut<1024, 8>>();
    if (e != cudaSuccess) return e;
    return set_pass_attrs<2048, 4, false, SIGN, SeqSrc<2048, 4>, SeqOut<2048, 4>>();
}

bool fft_c2c_single_pass(int64_t N) { return N == 1024 || N == 2048; }

cudaError_t launch_fft_c2c_single(const float2 *x, float2 *y, int64_t N, int64_t batch, int sign, cudaStream_t st) {
    if (N == 1024) return sign < 0 ? run_c2c_single<1024, -1>(x, y, batch, st) : run_c2c_single<1024, +1>(x, y, batch, st);
    if (N == 2048) return sign < 0 ? run_c2c_single<2048, -1>(x, y, batch, st) : run_c2c_single<2048, +1>(x, y, batch, st);
    return cudaErrorInvalidValue;
}

static int ilog2_i64(int64_t n) {
    int r = 0;
    while ((int64_t)1 << (r + 1) <= n) ++r;
    return r;
}

MF_DEBUG_READER(dbg_read_prep)

cudaError_t launch_forward_fft(const float *s, int64_t N, float2 *exch, float2 *X, cudaStream_t st) {
    FwdOp op{s, exch, X, ilog2_i64(N), st};
    return dispatch_split(op.log2N, op);
}

cudaError_t launch_fft_c2c(const float2 *x, float2 *y, int64_t N, int batch, int sign, float2 *exch,
                           cudaStream_t st) {
    const int lg = ilog2_i64(N);
    if (sign < 0) {
        C2COp<-1> op{x, y, exch, batch, st};
        return dispatch_split(lg, op);
    }
    C2COp<+1> op{x, y, exch, batch, st};
    return dispatch_split(lg, op);
}

cudaError_t prep_kernel_attributes() {
    {
        cudaError_t e0 = init_pass_tables();
        if (e0 != cudaSuccess) return e0;
    }
    for (int lg = 10; lg <= 22; ++lg) {
        C2CAttrOp<-1> a;
        C2CAttrOp<+1> b;
        cudaError_t e = dispatch_split(lg, a);
        if (e == cudaSuccess) e = dispatch_split(lg, b);
        if (e != cudaSuccess) return e;
    }
    for (int lg = 10; lg <= 22; ++lg) {
        FwdAttrOp op;
        cudaError_t e = dispatch_split(lg, op);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = c2c_single_attrs<-1>();
    if (e == cudaSuccess) e = c2c_single_attrs<+1>();
    return e;
}

// q_k = f^(-7/3)/S_k for 1 <= k < N/2, q_0 = 0.  Eq. (2) is evaluated as
// S0 * B(f) with the bracket B and the powers of f in FP32 (powf), the
// quotient scaled by 1/S0 in FP64; a caller table is used in FP64.
__device__ __forceinline__ float psd_eq2_bracket(float f, float f0) {
    const float x = f / f0;
    return powf(4.49f * x, -56.0f) + 0.16f * powf(x, -4.52f) + 0.52f + 0.32f * x * x;
}

__global__ void k_psd_weights(const double *__restrict__ psd, double f0, double S0, int64_t N, double fs,
                              double *__restrict__ q) {
    const int64_t half = N / 2;
    const double df = fs / (double)N;
    const double inv_S0 = 1.0 / S0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < half; k += (int64_t)gridDim.x * blockDim.x) {
        if (k == 0) { q[0] = 0.0; continue; }
        const double f = (double)k * df;
        const float p73 = powf((float)f, -7.0f / 3.0f);
        if (psd) q[k] = (double)p73 / psd[k];
        else q[k] = (double)(p73 / psd_eq2_bracket((float)f, (float)f0)) * inv_S0;
    }
}

cudaError_t launch_psd_weights(const float2 *X, const double *psd, double psd_f0, double psd_S0, int64_t N,
                               double fs, double *q, cudaStream_t st) {
    (void)X;
    const int64_t half = N / 2;
    int blocks = (int)((half + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_psd_weights<<<blocks, 256, 0, st>>>(psd, psd_f0, psd_S0, N, fs, q);
    return cudaGetLastError();
}

// ---- deterministic FP64 exclusive prefix: P[0] = 0, P[i+1] = P[i] + q[i] ----
constexpr int kScanThreads = 256;
constexpr int kScanPer = 32;
constexpr int kScanBlock = kScanThreads * kScanPer;

int64_t prefix_block_tmp_count(int64_t n) { return (n + kScanBlock - 1) / kScanBlock + 1; }

__device__ double block_exclusive_scan_f64(double x, double *sh) {
    // Hillis-Steele over 256 threads (fixed order -> deterministic)
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
        const double y = threadIdx.x >= (unsigned)o ? sh[threadIdx.x - o] : 0.0;
        __syncthreads();
        sh[threadIdx.x] += y;
        __syncthreads();
    }
    const double incl = sh[threadIdx.x];
    __syncthreads();
    return incl - x;
}

__global__ void k_scan_partials(const double *__restrict__ q, int64_t n, double *__restrict__ bsum) {
    __shared__ double sh[kScanThreads];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanPer;
    double s = 0.0;
    for (int i = 0; i < kScanPer; ++i) {
        const int64_t k = base + i;
        if (k < n) s += q[k];
    }
    const double ex = block_exclusive_scan_f64(s, sh);
    if (threadIdx.x == kScanThreads - 1) bsum[blockIdx.x] = ex + s;
}

__global__ void k_scan_blocksums(double *bsum, int nb) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double run = 0.0;
    for (int b = 0; b < nb; ++b) {
        const double v = bsum[b];
        bsum[b] = run;
        run += v;
    }
    bsum[nb] = run;
}

__global__ void k_scan_final(const double *__restrict__ q, int64_t n, const double *__restrict__ bsum,
                             double *__restrict__ P) {
    __shared__ double sh[kScanThreads];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanPer;
    double s = 0.0;
    for (int i = 0; i < kScanPer; ++i) {
        const int64_t k = base + i;
        if (k < n) s += q[k];
    }
    double run = bsum[blockIdx.x] + block_exclusive_scan_f64(s, sh);
    if (blockIdx.x == 0 && threadIdx.x == 0) P[0] = 0.0;
    for (int i = 0; i < kScanPer; ++i) {
        const int64_t k = base + i;
        if (k < n) {
            run += q[k];
            P[k + 1] = run;
        }
    }
}

cudaError_t launch_prefix_f64(const double *q, int64_t n, double *P, double *block_tmp, cudaStream_t st) {
    const int nb = (int)((n + kScanBlock - 1) / kScanBlock);
    k_scan_partials<<<nb, kScanThreads, 0, st>>>(q, n, block_tmp);
    k_scan_blocksums<<<1, 32, 0, st>>>(block_tmp, nb);
    k_scan_final<<<nb, kScanThreads, 0, st>>>(q, n, block_tmp, P);
    return cudaGetLastError();
}

// W_k = alpha f^(-7/6) dt conj(X_k)/S_k for 1 <= k < N/2, W_0 = 0; the real
// factor a_k = alpha f^(-7/6) dt / S_k depends on the PSD only and is kept
// in fac (when not NULL) so that new samples need only W_k = a_k conj(X_k)
__global__ void k_weight_data(const float2 *__restrict__ X, const double *__restrict__ psd, double f0, double S0,
                              int64_t N, double fs, const double *__restrict__ P, SegConsts *consts,
                              float2 *__restrict__ W, float *__restrict__ fac) {
    const int64_t half = N / 2;
    const double df = fs / (double)N, dt = 1.0 / fs;
    const double Ptot = P[half];
    const double alpha = sqrt(4.0 * df / Ptot);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        consts->P_tot = Ptot;
        consts->alpha = alpha;
    }
    const float a_eq2 = (float)(alpha * dt / S0);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < half; k += (int64_t)gridDim.x * blockDim.x) {
        if (k == 0) {
            W[0] = make_float2(0.f, 0.f);
            if (fac) fac[0] = 0.f;
            continue;
        }
        const float f = (float)((double)k * df);
        const float p76 = powf(f, -7.0f / 6.0f);
        const float a = psd ? (float)(alpha * dt / psd[k]) * p76 : a_eq2 * (p76 / psd_eq2_bracket(f, (float)f0));
        const float2 x = X[k];
        W[k] = make_float2(a * x.x, -a * x.y);
        if (fac) fac[k] = a;
    }
}

cudaError_t launch_weight_data(const float2 *X, const double *psd, double psd_f0, double psd_S0, int64_t N,
                               double fs, const double *P, SegConsts *consts, float2 *W, float *fac,
                               cudaStream_t st) {
    const int64_t half = N / 2;
    int blocks = (int)((half + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_weight_data<<<blocks, 256, 0, st>>>(X, psd, psd_f0, psd_S0, N, fs, P, consts, W, fac);
    return cudaGetLastError();
}

// W_k = a_k conj(X_k) with the segment's kept factors (new samples, same PSD)
__global__ void k_apply_weights(const float2 *__restrict__ X, const float *__restrict__ fac, int64_t half,
                                float2 *__restrict__ W) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < half; k += (int64_t)gridDim.x * blockDim.x) {
        const float a = fac[k];
        const float2 x = X[k];
        W[k] = make_float2(a * x.x, -a * x.y);
    }
}

cudaError_t launch_apply_weights(const float2 *X, const float *fac, int64_t N, float2 *W, cudaStream_t st) {
    const int64_t half = N / 2;
    int blocks = (int)((half + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_apply_weights<<<blocks, 256, 0, st>>>(X, fac, half, W);
    return cudaGetLastError();
}

}  // namespace mf
