// mf_passes.cuh -- the two passes of the four-step FFT as kernels templated on
// their data source and sink, plus the generic sources/sinks used by segment
// preparation and synthesis.  Geometry: N = N1 * N2 with N2 = 2^floor(log2 N / 2)
// the pass-1 (column) length and N1 = N / N2 the pass-2 (row) length;
// spectrum index k = k1 + N1 k2, time index j = j2 + N2 j1, exchange layout
// E[j2 * N1 + k1] (row j2 contiguous).
#pragma once
#include "mf_fft.cuh"
#include "mf_internal.h"

namespace mf {

template <int L>
__host__ __device__ constexpr int seqs_per_cta(int other) {
    return (8192 / L) < other ? (8192 / L) : other;
}

template <int L, int C>
__host__ __device__ constexpr size_t pass_data_bytes() {
    return (size_t)C * SeqStride<L, C>::value * sizeof(float2);
}
// data area, then the twiddle table, then the source's scratch
template <int L, int C, class Src>
__host__ __device__ constexpr size_t pass_smem_bytes() {
    return pass_data_bytes<L, C>() + (size_t)TwTable<L>::SIZE * sizeof(float2) + Src::kScratchBytes;
}

// Every source and sink is constructed with (params, tile, unit, slot): tile
// = which group of C sequences, unit = (template, segment) unit index, slot =
// which batch entry of the ring buffers it reads or writes; a source also gets
// Src::kScratchBytes of shared memory of its own.
// Generic pass kernel: grid.x = N_other / C tiles, grid.y = batch
// (unit = unit0 + blockIdx.y, slot = blockIdx.y).
template <int L, int C, bool SEQ_FAST, int SIGN, class Src, class Snk>
__global__ void __launch_bounds__(C *(L / 32), (C * (L / 32) >= 256) ? 2 : 1)
    k_fft_pass(typename Src::Params sp, typename Snk::Params kp, int unit0) {
    extern __shared__ float2 smem[];
    float2 *tw = smem + pass_data_bytes<L, C>() / sizeof(float2);
    fill_twiddles<L>(tw);
    Src src(sp, blockIdx.x, unit0 + blockIdx.y, blockIdx.y, tw + TwTable<L>::SIZE);
    Snk snk(kp, blockIdx.x, unit0 + blockIdx.y, blockIdx.y);
    cta_fft<L, C, SEQ_FAST, SIGN>(smem, tw, src, snk);
    snk.finish(smem);
}

template <int L, int C, bool SEQ_FAST, int SIGN, class Src, class Snk>
cudaError_t set_pass_attrs() {
    return cudaFuncSetAttribute(k_fft_pass<L, C, SEQ_FAST, SIGN, Src, Snk>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)pass_smem_bytes<L, C, Src>());
}

template <int L, int C, bool SEQ_FAST, int SIGN, class Src, class Snk>
cudaError_t run_pass(dim3 grid, const typename Src::Params &sp, const typename Snk::Params &kp,
                     cudaStream_t st, int unit0 = 0) {
    k_fft_pass<L, C, SEQ_FAST, SIGN, Src, Snk>
        <<<grid, C * (L / 32), pass_smem_bytes<L, C, Src>(), st>>>(sp, kp, unit0);
    return cudaGetLastError();
}

// Calls op.template run<N2, N1>() for the split of N = 2^log2N.
template <class Op>
cudaError_t dispatch_split(int log2N, Op &op) {
    switch (log2N) {
        case 10: return op.template run<32, 32>();
        case 11: return op.template run<32, 64>();
        case 12: return op.template run<64, 64>();
        case 13: return op.template run<64, 128>();
        case 14: return op.template run<128, 128>();
        case 15: return op.template run<128, 256>();
        case 16: return op.template run<256, 256>();
        case 17: return op.template run<256, 512>();
        case 18: return op.template run<512, 512>();
        case 19: return op.template run<512, 1024>();
        case 20: return op.template run<1024, 1024>();
        case 21: return op.template run<1024, 2048>();
        case 22: return op.template run<2048, 2048>();
        default: return cudaErrorInvalidValue;
    }
}

// op.template run<N2, N1>() for the split N = N1 * N2 with N2 = 2^log2N2:
// the balanced split of dispatch_split or the alternative one.
template <class Op>
cudaError_t dispatch_split2(int log2N, int log2N2, Op &op) {
    if (log2N2 == log2_n2(log2N)) return dispatch_split(log2N, op);
    if (log2N2 != alt_log2n2(log2N)) return cudaErrorInvalidValue;
    switch (log2N) {
        case 18: return op.template run<256, 1024>();
        case 19: return op.template run<1024, 512>();
        case 20: return op.template run<512, 2048>();
        case 21: return op.template run<2048, 1024>();
        case 22: return op.template run<1024, 4096>();
        default: return cudaErrorInvalidValue;
    }
}

// Deferred release of a work counter by thread 0 (persistent scheduler): the
// device-scope fence orders the block's writes of the previous item, which
// thread 0 observed through the block barrier that ended that item, before
// the increment.  Called right after the next item's loads are issued, so the
// fence's wait overlaps the load latency thread 0 has to wait for anyway.
__device__ __forceinline__ void release_hook(unsigned *ctr) {
    if (ctr != nullptr && threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
    }
}

// ---------------------------------------------------------------------------
// Column (pass-1) sources.  Sequence seq of CTA blockIdx.x is column
// k1 = blockIdx.x * C + seq; element n of it is spectrum entry k1 + N1 n.
// ---------------------------------------------------------------------------
template <int L, int C, bool HALF_ZERO, int LG1>
struct ColComplexSrc {      // X[k], zero for k >= N/2 when HALF_ZERO; LG1 = log2 N1
    static constexpr bool kHalfZero = HALF_ZERO;
    static constexpr size_t kScratchBytes = 0;
    struct Params { const float2 *X; int log2N1; int64_t batch_stride; };
    const Params &p;
    const int tile, slot;
    __device__ ColComplexSrc(const Params &pp, int tl, int, int sl, void *) : p(pp), tile(tl), slot(sl) {}
    __device__ __forceinline__ void load(int seq, int t, float2 *v) const {
        const float2 *X = p.X + (int64_t)slot * p.batch_stride;
        const int k1 = tile * C + seq;
        constexpr int T = L / 32;
        constexpr int NR = HALF_ZERO ? 16 : 32;
        const float2 *col = X + k1 + ((int64_t)t << LG1);
#pragma unroll
        for (int r = 0; r < NR; ++r) v[r] = col[(int64_t)r * T << LG1];
    }
};

template <int L, int C, int LG1>
struct ColRealSrc {         // real samples s[n] (imaginary part zero)
    static constexpr bool kHalfZero = false;
    static constexpr size_t kScratchBytes = 0;
    struct Params { const float *s; int log2N1; };
    const Params &p;
    const int tile;
    __device__ ColRealSrc(const Params &pp, int tl, int, int, void *) : p(pp), tile(tl) {}
    __device__ __forceinline__ void load(int seq, int t, float2 *v) const {
        const int k1 = tile * C + seq;
        constexpr int T = L / 32;
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = make_float2(p.s[k1 + ((t + r * T) << LG1)], 0.f);
    }
};

// Roots exp(+2 pi i m / 2^p), p = 10 .. 22, for the four-step twiddles of the
// exchange sinks, whose exponents stay below N / 32: per p a low table
// lo[j] = e^{2 pi i j / 2^p}, j < 1024, then a high table
// hi[i] = e^{2 pi i 1024 i / 2^p}, i < max(1, 2^(p - 15)); a root is
// hi[m >> 10] lo[m & 1023].  Entries are FP64 sincospi of exact arguments
// rounded to FP32 (once per device, per translation unit like the Stockham
// tables, by init_pass_tables).
__host__ __device__ constexpr int fs_hi_count(int p) { return p > 15 ? 1 << (p - 15) : 1; }
// start of the tables of p: the lengths 1024 + fs_hi_count(q) summed over q = 10 .. p - 1
__host__ __device__ constexpr int fs_offset(int p) {
    return 1024 * (p - 10) + (p - 10 < 6 ? p - 10 : 6) + (p >= 17 ? (1 << (p - 15)) - 2 : 0);
}
constexpr int kFsTotal = fs_offset(23);
static_assert(fs_offset(11) == 1025 && fs_offset(17) == fs_offset(16) + 1026 && fs_offset(18) == fs_offset(17) + 1028 &&
                  fs_offset(23) == fs_offset(22) + 1024 + 128,
              "root table layout");
static __device__ float2 g_fs_roots[kFsTotal];

static __global__ void k_init_fs_roots() {
    for (int p = 10; p <= 22; ++p) {
        float2 *tab = g_fs_roots + fs_offset(p);   // lo then hi
        const double P = (double)(1 << p);
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < 1024 + fs_hi_count(p); j += gridDim.x * blockDim.x) {
            const double m = j < 1024 ? (double)j : 1024.0 * (double)(j - 1024);
            double sn, cs;
            sincospi(2.0 * m / P, &sn, &cs);
            tab[j] = make_float2((float)cs, (float)sn);
        }
    }
}

// exp(SIGN 2 pi i m / 2^p) for 0 <= m < 2^(p - 5), from lo = g_fs_roots + fs_offset(p)
template <int SIGN>
__device__ __forceinline__ float2 fs_root(const float2 *lo, uint32_t m) {
    const float2 a = __ldg(&lo[1024 + (m >> 10)]), b = __ldg(&lo[m & 1023u]);
    const float2 r = make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
    return make_float2(r.x, SIGN > 0 ? r.y : -r.y);
}

// The Stockham tables and the four-step roots of this translation unit (every
// unit that launches kernels with an ExchSink calls this once per device).
static inline cudaError_t init_pass_tables() {
    k_init_fs_roots<<<8, 256>>>();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return init_twiddle_tables();
}

// Column sink: multiply by the four-step twiddle exp(SIGN 2 pi i j2 k1 / N)
// and write E[j2 * N1 + k1] (batch blockIdx.y at E + blockIdx.y * N).
template <int L, int C, int SIGN, int LG1>
struct ExchSink {
    struct Params { float2 *E; int log2N1; int log2N; };
    const Params &p;
    const int tile, slot;
    __device__ ExchSink(const Params &pp, int tl, int, int sl) : p(pp), tile(tl), slot(sl) {}
    template <int R>
    __device__ __forceinline__ void store(int seq, int b, int stride, const float2 *v) const {
        const int k1 = tile * C + seq;
        float2 *E = p.E + ((int64_t)slot << p.log2N) + ((int64_t)b << LG1) + k1;   // row j2 = b
        if (!MF_DBG(k1 < (1 << LG1) && b + (R - 1) * stride < (1 << (p.log2N - LG1)) && p.log2N >= 10 &&
                        p.log2N <= 22 && (int64_t)max(b, stride) * k1 < ((int64_t)1 << (p.log2N - 5)),
                    kDbgExch))
            return;
        const float2 *roots = g_fs_roots + fs_offset(p.log2N);   // b k1, stride k1 < N / 32
        float2 w = fs_root<SIGN>(roots, (uint32_t)(b * k1));
        const float2 step = fs_root<SIGN>(roots, (uint32_t)(stride * k1));
#pragma unroll
        for (int r = 0; r < R; ++r) {
            __stcg(&E[((int64_t)r * stride) << LG1], cmul(v[r], w));   // row j2 = b + r stride
            if (r + 1 < R) w = cmul(w, step);
        }
    }
    __device__ __forceinline__ void finish(float2 *) const {}
};

// ---------------------------------------------------------------------------
// Row (pass-2) source and generic sinks.  Sequence seq of CTA blockIdx.x is
// row j2 = blockIdx.x * C + seq of E; its element k1 is E[j2 * N1 + k1].
// ---------------------------------------------------------------------------
template <int L, int C>
struct RowSrc {
    static constexpr bool kHalfZero = false;
    static constexpr size_t kScratchBytes = 0;
    struct Params { const float2 *E; int log2N1; int log2N; };
    const Params &p;
    const int tile, slot;
    unsigned *rel = nullptr;   // deferred release (persistent scheduler)
    __device__ RowSrc(const Params &pp, int tl, int, int sl, void *) : p(pp), tile(tl), slot(sl) {}
    __device__ __forceinline__ void load(int seq, int t, float2 *v) const {
        const float2 *E = p.E + ((int64_t)slot << p.log2N);
        const int j2 = tile * C + seq;
        const float2 *row = E + ((int64_t)j2 << p.log2N1);
        constexpr int T = L / 32;
        if (!MF_DBG(j2 < (1 << (p.log2N - p.log2N1)) && p.log2N1 == cx_ilog2(L), kDbgExch)) row = E;
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = __ldcg(&row[t + r * T]);
        release_hook(rel);
    }
};

// out[j2 + N2 j1] = v for indices < limit
template <int L, int C>
struct RowComplexOut {
    struct Params { float2 *out; int log2N2; int64_t limit; };
    const Params &p;
    const int tile;
    __device__ RowComplexOut(const Params &pp, int tl, int, int) : p(pp), tile(tl) {}
    template <int R>
    __device__ __forceinline__ void store(int seq, int b, int stride, const float2 *v) const {
        const int j2 = tile * C + seq;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t j = j2 + ((int64_t)(b + r * stride) << p.log2N2);
            if (j < p.limit) p.out[j] = v[r];
        }
    }
    __device__ __forceinline__ void finish(float2 *) const {}
};

// out[slot * out_stride + j2 + N2 j1] = v for every j.  The CTA owns C
// consecutive rows j2, so each j1 is C consecutive outputs; every thread
// parks its outputs in its sequence's shared-memory row (free once every
// thread of the sequence has read its last stage: the warp for rows of up to
// 1024 points, the CTA for 2048) and finish() writes the C x L tile with
// consecutive threads on consecutive outputs.  Longer rows would store
// element by element.
template <int L, int C>
struct RowTileOut {
    static constexpr bool kTile = (L / 32) <= 64;
    struct Params { float2 *out; int log2N2; int64_t out_stride; };
    const Params &p;
    const int tile, slot;
    __device__ RowTileOut(const Params &pp, int tl, int, int sl) : p(pp), tile(tl), slot(sl) {}
    __device__ __forceinline__ float2 *row(int seq) const {
        extern __shared__ float2 rto_smem[];
        return rto_smem + seq * SeqStride<L, C>::value;
    }
    template <int R>
    __device__ __forceinline__ void store(int seq, int b, int stride, const float2 *v) const {
        if constexpr (kTile) {
            float2 *r0 = row(seq);
            if constexpr (L / 32 <= 32) __syncwarp();   // the sequence's threads have read their last stage
            else __syncthreads();                        // (two warps per 2048-point sequence; all threads get here once)
#pragma unroll
            for (int r = 0; r < R; ++r) r0[b + r * stride] = v[r];
        } else {
            float2 *o = p.out + slot * p.out_stride + tile * C + seq;
#pragma unroll
            for (int r = 0; r < R; ++r) o[(int64_t)(b + r * stride) << p.log2N2] = v[r];
        }
    }
    __device__ __forceinline__ void finish(float2 *) const {
        if constexpr (kTile) {
            __syncthreads();
            float2 *o = p.out + slot * p.out_stride + tile * C;
            for (int idx = threadIdx.x; idx < C * L; idx += blockDim.x) {
                const int seq = idx % C, j1 = idx / C;
                __stcs(&o[seq + ((int64_t)j1 << p.log2N2)], row(seq)[j1]);
            }
        }
    }
};

// s[j2 + N2 j1] = scale * Re(v)
template <int L, int C>
struct RowRealOut {
    struct Params { float *s; int log2N2; float scale; };
    const Params &p;
    const int tile;
    __device__ RowRealOut(const Params &pp, int tl, int, int) : p(pp), tile(tl) {}
    template <int R>
    __device__ __forceinline__ void store(int seq, int b, int stride, const float2 *v) const {
        const int j2 = tile * C + seq;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t j = j2 + ((int64_t)(b + r * stride) << p.log2N2);
            p.s[j] = p.scale * v[r].x;
        }
    }
    __device__ __forceinline__ void finish(float2 *) const {}
};

}  // namespace mf
