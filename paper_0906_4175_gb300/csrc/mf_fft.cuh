// mf_fft.cuh -- FP32 complex FFT building blocks for sm_103a.
//
// The inverse FFT of Eq. (1) (and the forward FFT of the data) is a four-step
// transform N = N1 * N2: pass 1 runs N1 column FFTs of length N2 (stride N1 in
// the spectrum), multiplies by the inter-pass twiddles exp(+-2 pi i j2 k1 / N)
// and writes one complex64 exchange array; pass 2 runs N2 row FFTs of length
// N1.  Each CTA transforms C sequences of length L = 2^m (32 <= L <= 4096) held
// in shared memory, with a Stockham autosort schedule (the index mapping of
// Govindaraju et al., "High Performance Discrete Fourier Transforms on Graphics
// Processors", SC 2008): stage radices (32, min(32, L/32), L/1024), every
// thread holding 32 complex values in registers per stage, radix-32/16/8/4/2
// butterflies fully unrolled with compile-time twiddle constants.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mf {

// ----------------------------------------------------------------------------
// Compile-time cos/sin of 2 pi num/den: exact integer reduction to the first
// octant, then Taylor series in double (|x| <= pi/4, 14 terms: < 1e-30).
// ----------------------------------------------------------------------------
constexpr double kPi = 3.14159265358979323846264338327950288;

struct CxCS { double c, s; };

__host__ __device__ constexpr double cx_sin_series(double x) {
    double t = x, s = x;
    for (int n = 1; n < 14; ++n) { t *= -x * x / ((2.0 * n) * (2.0 * n + 1.0)); s += t; }
    return s;
}
__host__ __device__ constexpr double cx_cos_series(double x) {
    double t = 1.0, s = 1.0;
    for (int n = 1; n < 14; ++n) { t *= -x * x / ((2.0 * n - 1.0) * (2.0 * n)); s += t; }
    return s;
}
__host__ __device__ constexpr CxCS cx_sincos_turn(long long num, long long den) {
    long long m = num % den;
    if (m < 0) m += den;
    long long q = (4 * m) / den;          // quadrant
    long long r = 4 * m - q * den;        // angle within quadrant = (pi/2) r / den
    double c = 0.0, s = 0.0;
    if (2 * r <= den) {
        double x = (kPi / 2.0) * (double)r / (double)den;
        c = cx_cos_series(x); s = cx_sin_series(x);
    } else {
        double y = (kPi / 2.0) * (double)(den - r) / (double)den;
        c = cx_sin_series(y); s = cx_cos_series(y);
    }
    if (q == 0) return CxCS{c, s};
    if (q == 1) return CxCS{-s, c};
    if (q == 2) return CxCS{-c, -s};
    return CxCS{s, -c};
}

__host__ __device__ constexpr int cx_ilog2(long long x) {
    int r = 0;
    while (x > 1) { x >>= 1; ++r; }
    return r;
}

// ----------------------------------------------------------------------------
// complex helpers
// ----------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 czero() { return make_float2(0.f, 0.f); }

// x * exp(SIGN * 2 pi i Q / R), Q and R compile-time
template <int Q, int R, int SIGN>
__device__ __forceinline__ float2 tw_const(float2 x) {
    constexpr long long g = Q % R;
    if constexpr (g == 0) {
        return x;
    } else if constexpr (4 * g == R) {                  // exp(+-i pi/2) = +-i
        return SIGN > 0 ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
    } else if constexpr (2 * g == R) {                  // -1
        return make_float2(-x.x, -x.y);
    } else if constexpr (4 * g == 3 * R) {              // exp(+-3 i pi/2) = -+i
        return SIGN > 0 ? make_float2(x.y, -x.x) : make_float2(-x.y, x.x);
    } else {
        constexpr CxCS w = cx_sincos_turn(SIGN * g, R);
        constexpr float c = (float)w.c;
        constexpr float s = (float)w.s;
        return make_float2(fmaf(c, x.x, -s * x.y), fmaf(c, x.y, s * x.x));
    }
}

// ----------------------------------------------------------------------------
// In-register DFT of length R (natural order in and out), radix-2 DIT
// recursion with compile-time twiddles:  X_q = sum_r v_r exp(SIGN 2 pi i r q / R)
// ----------------------------------------------------------------------------
__host__ __device__ constexpr double cx_abs(double x) { return x < 0 ? -x : x; }

// Radix-2 combine  v[Q] = e[Q] + w o[Q],  v[Q + R/2] = e[Q] - w o[Q],
// w = exp(SIGN 2 pi i Q / R).  A general w = c + i s is applied in the
// multiply-add form of Linzer & Feig (1993): w o = c (o (1 + i s/c)) when
// |c| >= |s|, else s (o (c/s + i)); the inner product takes 2 FMAs and the
// scaled add/subtract 4, i.e. 6 instead of 8 instructions.
template <int R, int SIGN, int Q>
struct Combine {
    static __device__ __forceinline__ void run(float2 *v, const float2 *e, const float2 *o) {
        if constexpr (Q < R / 2) {
            constexpr long long g = Q % R;
            if constexpr (g == 0 || 4 * g == R) {
                const float2 t = tw_const<Q, R, SIGN>(o[Q]);
                v[Q] = cadd(e[Q], t);
                v[Q + R / 2] = csub(e[Q], t);
            } else {
                constexpr CxCS w = cx_sincos_turn(SIGN * g, R);
                float2 b;
                float k;
                if constexpr (cx_abs(w.c) >= cx_abs(w.s)) {
                    constexpr float tt = (float)(w.s / w.c);
                    constexpr float kc = (float)w.c;
                    b = make_float2(fmaf(-tt, o[Q].y, o[Q].x), fmaf(tt, o[Q].x, o[Q].y));
                    k = kc;
                } else {
                    constexpr float ct = (float)(w.c / w.s);
                    constexpr float ks = (float)w.s;
                    b = make_float2(fmaf(ct, o[Q].x, -o[Q].y), fmaf(ct, o[Q].y, o[Q].x));
                    k = ks;
                }
                v[Q] = make_float2(fmaf(k, b.x, e[Q].x), fmaf(k, b.y, e[Q].y));
                v[Q + R / 2] = make_float2(fmaf(-k, b.x, e[Q].x), fmaf(-k, b.y, e[Q].y));
            }
            Combine<R, SIGN, Q + 1>::run(v, e, o);
        }
    }
};

template <int R, int SIGN>
struct Dft {
    static __device__ __forceinline__ void run(float2 *v) {
        if constexpr (R == 1) {
            return;
        } else if constexpr (R == 2) {
            float2 a = v[0], b = v[1];
            v[0] = cadd(a, b);
            v[1] = csub(a, b);
        } else {
            float2 e[R / 2], o[R / 2];
#pragma unroll
            for (int i = 0; i < R / 2; ++i) { e[i] = v[2 * i]; o[i] = v[2 * i + 1]; }
            Dft<R / 2, SIGN>::run(e);
            Dft<R / 2, SIGN>::run(o);
            Combine<R, SIGN, 0>::run(v, e, o);
        }
    }
};

// 32-point DFT whose inputs v[16..31] are zero (upper half of a one-sided
// spectrum): even outputs are the 16-point DFT of v, odd outputs the 16-point
// DFT of v_r exp(SIGN 2 pi i r/32).
template <int SIGN, int Q>
struct HalfZeroTw {
    static __device__ __forceinline__ void run(const float2 *v, float2 *b) {
        if constexpr (Q < 16) {
            b[Q] = tw_const<Q, 32, SIGN>(v[Q]);
            HalfZeroTw<SIGN, Q + 1>::run(v, b);
        }
    }
};
template <int SIGN>
__device__ __forceinline__ void dft32_halfzero(float2 *v) {
    float2 a[16], b[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = v[i];
    HalfZeroTw<SIGN, 0>::run(v, b);
    Dft<16, SIGN>::run(a);
    Dft<16, SIGN>::run(b);
#pragma unroll
    for (int p = 0; p < 16; ++p) { v[2 * p] = a[p]; v[2 * p + 1] = b[p]; }
}

// v[r] *= w^r for r = 1..R-1 (w^r by repeated multiplication)
template <int R>
__device__ __forceinline__ void twiddle_powers(float2 *v, float2 w) {
    float2 cur = w;
#pragma unroll
    for (int r = 1; r < R; ++r) {
        v[r] = cmul(v[r], cur);
        if (r + 1 < R) cur = cmul(cur, w);
    }
}

// exp(SIGN * 2 pi i num / den) for den a power of two (FP32, argument exact)
template <int SIGN>
__device__ __forceinline__ float2 unit_root(uint32_t num, uint32_t log2den) {
    uint32_t m = num & ((1u << log2den) - 1u);
    float a = __uint_as_float((uint32_t)(127 - (int)log2den + 1) << 23) * (float)m;  // 2 m / den, exact
    float s, c;
    sincospif(a, &s, &c);
    return make_float2(c, SIGN > 0 ? s : -s);
}

// ----------------------------------------------------------------------------
// Stockham schedule for one CTA: C sequences of length L, T = L/32 threads per
// sequence.  Shared memory holds the sequences with one pad element every 32
// and a column stride congruent to 2 mod 16 (float2 units) to spread banks.
// ----------------------------------------------------------------------------
template <int L>
struct FftShape {
    static_assert(L >= 32 && L <= 4096 && (L & (L - 1)) == 0, "L must be a power of two in [32, 4096]");
    static constexpr int T = L / 32;
    static constexpr int R1 = (L / 32 <= 32) ? L / 32 : 32;
    static constexpr int R2 = (L > 1024) ? L / 1024 : 1;
    static constexpr int NST = (L == 32) ? 1 : ((L <= 1024) ? 2 : 3);
    static constexpr int PADDED = L + L / 32;
    static constexpr int STRIDE = PADDED + ((2 - (PADDED % 16)) + 16) % 16;   // = 2 mod 16
};

__device__ __forceinline__ int spad(int m) { return m + (m >> 5); }

// Stride (float2 units) between the C sequences of a CTA: the padded length
// rounded up to 16/C (mod 16), or to 1 (mod 16) for C >= 16.  A half-warp of
// a column pass holds C sequences x 16/C positions (sequence fastest), so its
// 8-byte accesses land on 16 different bank pairs; the same holds for the
// sinks' tile flushes (sequence fastest).  For C = 8 this is the 2 (mod 16)
// of FftShape::STRIDE.
template <int L, int C>
struct SeqStride {
    static constexpr int PADDED = FftShape<L>::PADDED;
    static constexpr int RES = C >= 16 ? 1 : 16 / C;
    static constexpr int value = PADDED + ((RES - PADDED % 16) + 16) % 16;
};

// Twiddle tables of the Stockham stages after stage 0, in shared memory:
// for a stage (Ns, R) the entries w[r * Ns + k] = exp(+2 pi i r k / (Ns R)),
// r < R, k < Ns (k fastest, so a warp reading one r hits consecutive words).
// Stage 1 has Ns = 32; stage 2 (L > 1024) has Ns = 1024.
template <int L>
struct TwTable {
    static constexpr int S1 = 32 * FftShape<L>::R1;                        // stage-1 entries
    static constexpr int S2 = (FftShape<L>::NST == 3) ? 1024 * FftShape<L>::R2 : 0;
    static constexpr int SIZE = (FftShape<L>::NST == 1) ? 0 : S1 + S2;
};

// Compute the table of an L-point FFT (all threads of the block).
template <int L>
__device__ __forceinline__ void compute_twiddles(float2 *tw) {
    using S = FftShape<L>;
    if constexpr (S::NST >= 2) {
        constexpr int LG1 = cx_ilog2(32 * S::R1);
        for (int m = threadIdx.x; m < TwTable<L>::S1; m += blockDim.x) {
            const int r = m >> 5, k = m & 31;
            tw[m] = unit_root<+1>((uint32_t)(r * k), LG1);
        }
    }
    if constexpr (S::NST == 3) {
        constexpr int LG2 = cx_ilog2(L);
        for (int m = threadIdx.x; m < TwTable<L>::S2; m += blockDim.x) {
            const int r = m >> 10, k = m & 1023;
            tw[TwTable<L>::S1 + m] = unit_root<+1>((uint32_t)(r * k), LG2);
        }
    }
}

// Sinks may define after_loads(): called by the last stage once this thread's
// shared-memory reads are issued and before its arithmetic (a warp-owned
// region can be refilled from there on).
template <class T, class = void>
struct has_after_loads { static constexpr bool value = false; };
template <class T>
struct has_after_loads<T, decltype((void)&T::after_loads, void())> { static constexpr bool value = true; };

// The tables of every length, computed once per device by init_twiddle_tables()
// (one copy per translation unit that launches FFT kernels), so that a CTA
// only copies its table into shared memory instead of evaluating it.
template <int L>
__host__ __device__ constexpr int tw_offset() {
    if constexpr (L <= 32) return 0;
    else return tw_offset<L / 2>() + TwTable<L / 2>::SIZE;
}
constexpr int kTwTotal = tw_offset<8192>();   // the tables of L = 64 .. 4096
static __device__ float2 g_tw_tables[kTwTotal];

template <int L>
__global__ void k_init_twiddles() {
    compute_twiddles<L>(g_tw_tables + tw_offset<L>());
}

static inline cudaError_t init_twiddle_tables() {
    k_init_twiddles<64><<<1, 256>>>();
    k_init_twiddles<128><<<1, 256>>>();
    k_init_twiddles<256><<<1, 256>>>();
    k_init_twiddles<512><<<1, 256>>>();
    k_init_twiddles<1024><<<1, 256>>>();
    k_init_twiddles<2048><<<1, 256>>>();
    k_init_twiddles<4096><<<1, 256>>>();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaDeviceSynchronize();
}

// Copy the table of an L-point FFT into shared memory (all threads of the
// block; callers synchronise before first use).
template <int L>
__device__ __forceinline__ void fill_twiddles(float2 *tw) {
    const float2 *src = g_tw_tables + tw_offset<L>();
    for (int m = threadIdx.x; m < TwTable<L>::SIZE; m += blockDim.x) tw[m] = __ldg(&src[m]);
}

// Barrier between the stages of one FFT: the whole CTA by default; kernels in
// which a smaller group of threads owns a sequence pass their own.
struct CtaSync {
    static __device__ __forceinline__ void sync() { __syncthreads(); }
};

// One Stockham stage reading from and (unless LAST) writing to shared memory.
// Ns = product of earlier radices; each thread runs 32/R butterflies b = t + i*T.
template <int L, int R, int Ns, int SIGN, bool LAST, class Snk, class Sync = CtaSync>
__device__ __forceinline__ void stockham_stage(float2 *sq, const float2 *tw, int seq, int t, Snk &snk) {
    constexpr int T = L / 32;
    constexpr int NB = 32 / R;
    constexpr int SPAN = L / R;
    float2 v[32];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int b = t + i * T;
#pragma unroll
        for (int r = 0; r < R; ++r) v[i * R + r] = sq[spad(b + r * SPAN)];
    }
    if constexpr (!LAST) Sync::sync();
    if constexpr (LAST && has_after_loads<Snk>::value) snk.after_loads();
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int b = t + i * T;
        const int k = b & (Ns - 1);
        if constexpr (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = tw[r * Ns + k];
                if (SIGN < 0) w.y = -w.y;
                v[i * R + r] = cmul(v[i * R + r], w);
            }
        }
        Dft<R, SIGN>::run(v + i * R);
        if constexpr (!LAST) {
            const int idxD = (b / Ns) * Ns * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) sq[spad(idxD + r * Ns)] = v[i * R + r];
        }
    }
    if constexpr (LAST) {
        // In the last stage Ns R = L, so output r of butterfly i is element
        // t + i T + r L/R = t + T (i + r NB): all 32 outputs of the thread go to
        // the sink in one call (outputs t + q T), whatever the radix.
        if constexpr (NB == 1) {
            snk.template store<32>(seq, t, T, v);
        } else {
            float2 o[32];
#pragma unroll
            for (int i = 0; i < NB; ++i)
#pragma unroll
                for (int r = 0; r < R; ++r) o[i + r * NB] = v[i * R + r];
            snk.template store<32>(seq, t, T, o);
        }
    }
    if constexpr (!LAST) Sync::sync();
}

// Last Stockham stage of a 1024-point sequence (radix 32 over Ns = 32) with
// the twiddles exp(SIGN 2 pi i r t / 1024) of rows r > 16 formed as
// w[r - 16] w[16]: only rows r <= 16 of the table are read, so a kernel short
// of shared memory can keep just those 17 rows.  Thread t reads elements
// t + 32 r and hands the 32-point DFT to the sink (outputs t + 32 r).
template <int SIGN, class Snk>
__device__ __forceinline__ void last_stage_1024_split(const float2 *sq, const float2 *tw, int seq, int t, Snk &snk) {
    float2 v[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = sq[spad(t + 32 * r)];
    float2 w16 = tw[16 * 32 + t];
    if (SIGN < 0) w16.y = -w16.y;
#pragma unroll
    for (int r = 1; r < 16; ++r) {
        float2 w = tw[r * 32 + t];
        if (SIGN < 0) w.y = -w.y;
        v[r] = cmul(v[r], w);
        v[r + 16] = cmul(v[r + 16], cmul(w, w16));
    }
    v[16] = cmul(v[16], w16);
    Dft<32, SIGN>::run(v);
    snk.template store<32>(seq, t, 32, v);
}

// Sources that define kSplitTw = true have their 1024-point transforms end
// with last_stage_1024_split, so that every kernel generating templates
// (whatever its shared-memory budget) rounds the same way.
template <class T, class = void>
struct uses_split_tw { static constexpr bool value = false; };
template <class T>
struct uses_split_tw<T, decltype((void)T::kSplitTw, void())> { static constexpr bool value = T::kSplitTw; };

// Full CTA FFT.  tw: the TwTable<L> twiddles in shared memory, filled and
// made visible before the call (or filled before it with no intervening
// shared-memory write, the first stage barrier publishes them).
// Src::load(seq, t, v) fills v[r] = x[t + r*T], r < 32
// (Src::kHalfZero: v[16..31] are zero and are not read).
// Snk::store<R>(seq, b, stride, v) receives outputs b + r*stride, r < R
// (the Stockham stages call it once per thread with R = 32, b = t, stride = T).
// The last stage does not synchronise: a sink that reuses shared memory
// afterwards must __syncthreads() first.
// smem: C * SeqStride<L, C>::value float2.  Must be called by all C*T threads.
template <int L, int C, bool SEQ_FAST, int SIGN, class Src, class Snk>
__device__ __forceinline__ void cta_fft(float2 *smem, const float2 *tw, Src &src, Snk &snk) {
    using S = FftShape<L>;
    constexpr int T = S::T;
    const int tid = threadIdx.x;
    const int seq = SEQ_FAST ? (tid % C) : (tid / T);
    const int t = SEQ_FAST ? (tid / C) : (tid % T);
    float2 *sq = smem + seq * SeqStride<L, C>::value;

    {
        float2 v[32];
        src.load(seq, t, v);
        if constexpr (Src::kHalfZero) dft32_halfzero<SIGN>(v);
        else Dft<32, SIGN>::run(v);
        if constexpr (S::NST == 1) {
            snk.template store<32>(seq, t, T, v);
            return;
        } else {
#pragma unroll
            for (int r = 0; r < 32; ++r) sq[spad(32 * t + r)] = v[r];
        }
    }
    __syncthreads();
    if constexpr (S::NST == 2) {
        if constexpr (L == 1024 && uses_split_tw<Src>::value) last_stage_1024_split<SIGN>(sq, tw, seq, t, snk);
        else stockham_stage<L, S::R1, 32, SIGN, true>(sq, tw, seq, t, snk);
    } else if constexpr (S::NST == 3) {
        stockham_stage<L, S::R1, 32, SIGN, false>(sq, tw, seq, t, snk);
        stockham_stage<L, S::R2, 32 * S::R1, SIGN, true>(sq, tw + TwTable<L>::S1, seq, t, snk);
    }
}

}  // namespace mf
