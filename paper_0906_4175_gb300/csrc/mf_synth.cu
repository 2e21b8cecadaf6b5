// mf_synth.cu -- seeded synthetic data for the filter: stationary Gaussian
// noise coloured by the Eq. (2) PSD (the paper's test data is coloured
// Gaussian noise, Sec. 3) plus frequency-domain injections of the 2PN
// templates, then a real inverse FFT:
//   s~_k = noise_scale sqrt(T S_k / 4) (g_{2k} + i g_{2k+1}),  k_lo <= k < N/2,
//   s~_k += snr / sqrt(4 df Q_i) f^(-7/6) e^{-i Psi_i(f_k)} e^{-2 pi i k j0_i / N} e^{i phi_i}
//          on injection i's band (Q_i = sum_band f^(-7/3)/S_k, so that the
//          injection's optimal SNR is snr),
//   s_n = 2 df Re sum_k s~_k e^{+2 pi i n k / N}.
#include "mf_passes.cuh"

namespace mf {

__device__ __forceinline__ double psd_eq2_s(double f, double f0, double S0) {
    const double x = f / f0;
    return S0 * (pow(4.49 * x, -56.0) + 0.16 * pow(x, -4.52) + 0.52 + 0.32 * x * x);
}

// injection record (doubles): c1 c2 c3 c5 k_lo k_hi j0 phi/(2 pi) snr
constexpr int kInjStride = 10;

__global__ void k_synth_spectrum(const double *__restrict__ g, int64_t N, double fs, double f_low,
                                 const double *__restrict__ psd, double f0, double S0,
                                 const double *__restrict__ inj, int n_inj, const double *__restrict__ P,
                                 double noise_scale, float2 *__restrict__ Y) {
    const int64_t half = N / 2;
    const double df = fs / (double)N, T = (double)N / fs;
    int64_t k_lo = (int64_t)ceil(f_low * (double)N / fs);
    if (k_lo < 1) k_lo = 1;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < half; k += (int64_t)gridDim.x * blockDim.x) {
        double re = 0.0, im = 0.0;
        if (k >= k_lo) {
            const double f = (double)k * df;
            const double S = psd ? psd[k] : psd_eq2_s(f, f0, S0);
            const double a = noise_scale * sqrt(T * S / 4.0);
            re = a * g[2 * k];
            im = a * g[2 * k + 1];
            for (int i = 0; i < n_inj; ++i) {
                const double *I = inj + (int64_t)i * kInjStride;
                const int64_t lo = (int64_t)I[4], hi = (int64_t)I[5];
                if (k < lo || k >= hi) continue;
                const double Q = P[hi] - P[lo];
                const double amp = I[8] / sqrt(4.0 * df * Q) * pow(f, -7.0 / 6.0);
                const double u = rcbrt(f), u2 = u * u, u3 = u2 * u, u5 = u3 * u2;
                const double psi = -0.125 + I[0] * u + I[1] * u2 + I[2] * u3 + I[3] * u5;
                const int64_t j0 = (int64_t)I[6];
                const int64_t kj = (k * j0) % N;
                double ph = -psi - (double)kj / (double)N + I[7];
                ph -= rint(ph);
                double s, c;
                sincospi(2.0 * ph, &s, &c);
                re += amp * c;
                im += amp * s;
            }
        }
        Y[k] = make_float2((float)re, (float)im);
    }
}

cudaError_t launch_synth_spectrum(const double *g, int64_t N, double fs, double f_low, const double *psd,
                                  double psd_f0, double psd_S0, const double *inj_dev, int64_t n_inj,
                                  const double *P, double noise_scale, float2 *Y, cudaStream_t st) {
    const int64_t half = N / 2;
    int blocks = (int)((half + 255) / 256);
    if (blocks > 8192) blocks = 8192;
    k_synth_spectrum<<<blocks, 256, 0, st>>>(g, N, fs, f_low, psd, psd_f0, psd_S0, inj_dev, (int)n_inj, P,
                                             noise_scale, Y);
    return cudaGetLastError();
}

namespace {
struct InvRealOp {
    const float2 *Y;
    float2 *exch;
    float *s;
    float scale;
    int log2N;
    cudaStream_t st;
    template <int N2, int N1>
    cudaError_t run() {
        constexpr int C1 = seqs_per_cta<N2>(N1);
        constexpr int C2 = seqs_per_cta<N1>(N2);
        const int log2N2 = log2_n2(log2N), log2N1 = log2N - log2N2;
        typename ColComplexSrc<N2, C1, true, cx_ilog2(N1)>::Params sp{Y, log2N1, 0};
        typename ExchSink<N2, C1, +1, cx_ilog2(N1)>::Params kp{exch, log2N1, log2N};
        cudaError_t e = run_pass<N2, C1, true, +1, ColComplexSrc<N2, C1, true, cx_ilog2(N1)>, ExchSink<N2, C1, +1, cx_ilog2(N1)>>(
            dim3(N1 / C1, 1), sp, kp, st);
        if (e != cudaSuccess) return e;
        typename RowSrc<N1, C2>::Params sp2{exch, log2N1, log2N};
        typename RowRealOut<N1, C2>::Params kp2{s, log2N2, scale};
        return run_pass<N1, C2, false, +1, RowSrc<N1, C2>, RowRealOut<N1, C2>>(dim3(N2 / C2, 1), sp2, kp2, st);
    }
};
struct InvAttrOp {
    template <int N2, int N1>
    cudaError_t run() {
        constexpr int C1 = seqs_per_cta<N2>(N1);
        constexpr int C2 = seqs_per_cta<N1>(N2);
        cudaError_t e = set_pass_attrs<N2, C1, true, +1, ColComplexSrc<N2, C1, true, cx_ilog2(N1)>, ExchSink<N2, C1, +1, cx_ilog2(N1)>>();
        if (e != cudaSuccess) return e;
        return set_pass_attrs<N1, C2, false, +1, RowSrc<N1, C2>, RowRealOut<N1, C2>>();
    }
};
}  // namespace

cudaError_t launch_inverse_real_fft(const float2 *Y, int64_t N, double scale, float2 *exch, float *s,
                                    cudaStream_t st) {
    int lg = 0;
    while (((int64_t)1 << (lg + 1)) <= N) ++lg;
    InvRealOp op{Y, exch, s, (float)scale, lg, st};
    return dispatch_split(lg, op);
}

cudaError_t synth_kernel_attributes() {
    {
        cudaError_t e0 = init_pass_tables();
        if (e0 != cudaSuccess) return e0;
    }
    for (int lg = 10; lg <= 22; ++lg) {
        InvAttrOp op;
        cudaError_t e = dispatch_split(lg, op);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace mf
