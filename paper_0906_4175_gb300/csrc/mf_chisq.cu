// mf_chisq.cu -- the chi^2 consistency test of Eq. (5) (Sec. 1.2) as a full
// time series, the computation the paper moved to the GPU: the band of
// Eq. (1) is split into p sub-bands of equal sigma^2 share, each sub-band's
// z_l(t) comes from its own inverse FFT, and
//   chi^2(t) = (p / sigma^2) sum_l |z_l(t) - z(t)/p|^2
//            = rho_scale^2 (p sum_l |raw_l(t)|^2 - |raw(t)|^2)     (sum_l z_l = z),
// with raw the pass-2 output of the filter (rho = |raw| rho_scale).
// Sub-band l is b_l <= k < b_{l+1}: b_0 = k_lo, b_p = k_hi and, for 0 < l < p,
// b_l is the smallest k with P[k] - P[k_lo] >= (l/p)(P[k_hi] - P[k_lo]), P the
// segment's FP64 prefix of f^(-7/3)/S (|h~|^2/S up to the amplitude).
// Each sub-band runs through the filter's own pass 1 (template generation on
// the sub-band only, column IFFTs) and a pass 2 whose sink accumulates
// |raw_l|^2 into the caller's output row; the last, full-band pass 2 turns
// the sum into chi^2.  Neither z_l nor z is stored.
#include <algorithm>

#include "mf_filter.cuh"

namespace mf {

// One block per chi^2 unit: the sub-band edges by binary search in P, then
// p + 1 copies of the unit's full-band UnitInfo (band l = [b_l, b_{l+1}),
// band p = the full band).  A template index outside the bank gives an empty
// band (the output row is zero).
__global__ void k_chisq_units(SegDev seg, const UnitInfo *__restrict__ all, int n_t, const int32_t *__restrict__ tmpl,
                              int n, int p, UnitInfo *__restrict__ out, int64_t *__restrict__ edges) {
    __shared__ int64_t b[kChisqMaxBands + 1];
    const int u = blockIdx.x;
    const int t = tmpl[u];
    UnitInfo full;
    if (t >= 0 && t < n_t) {
        full = all[t];
    } else {   // empty band on template 0's record (keeps every later read in range)
        full = all[0];
        full.k_hi = full.k_lo;
    }
    const int64_t lo = full.k_lo, hi = full.k_hi;
    const double P0 = seg.P[lo], Q = seg.P[hi] - P0;
    for (int l = threadIdx.x; l <= p; l += blockDim.x) {
        int64_t e;
        if (l == 0) {
            e = lo;
        } else if (l == p) {
            e = hi;
        } else {
            const double target = ((double)l / (double)p) * Q;
            int64_t a = lo, c = hi;   // smallest k in [a, c] with P[k] - P0 >= target
            while (a < c) {
                const int64_t m = a + ((c - a) >> 1);
                if (seg.P[m] - P0 >= target) c = m;
                else a = m + 1;
            }
            e = a;
        }
        b[l] = e;
        if (edges) edges[(int64_t)u * (p + 1) + l] = e;
    }
    __syncthreads();
    for (int l = threadIdx.x; l <= p; l += blockDim.x) {
        UnitInfo x = full;
        if (l < p) {
            x.k_lo = (int32_t)b[l];
            x.k_hi = (int32_t)b[l + 1];
        }
        out[(int64_t)l * n + u] = x;
    }
}

// pass-2 sinks.  The CTA owns rows j2 = tile C .. tile C + C - 1, i.e. C
// consecutive samples out of every N2, so per-element global accesses from
// the butterflies would touch one 32-byte sector per lane.  Each thread
// therefore parks |raw|^2 of its outputs in its sequence's shared-memory row
// (free once every thread of the sequence has read its last stage: the warp
// for rows of up to 1024 points, the CTA for 2048), and finish() moves the
// C x N1 tile to the unit's output row with the C consecutive samples of each
// j1 on consecutive threads.
template <int L, int C>
__device__ __forceinline__ float *chi_tile_row(int seq) {
    extern __shared__ float2 chi_smem[];
    return reinterpret_cast<float *>(chi_smem + seq * SeqStride<L, C>::value);
}

template <int L, int C>
__device__ __forceinline__ void chi_park(int seq, int b, int stride, const float2 *v, int R) {
    float *row = chi_tile_row<L, C>(seq);
    if constexpr (L / 32 <= 32) __syncwarp();   // the sequence's threads have read their last-stage inputs
    else __syncthreads();                        // (a 2048-point sequence spans two warps; every thread gets here once)
#pragma unroll 32
    for (int r = 0; r < R; ++r) row[b + r * stride] = fmaf(v[r].x, v[r].x, v[r].y * v[r].y);
}

// mode 0: acc = |raw|^2, 1: acc += |raw|^2, 2: acc = rs2 (p acc - |raw|^2).
// Rows of up to 2048 points go through the shared-memory tile; longer rows
// would update the output element by element from the butterflies.
template <int L, int C>
struct ChiSink {
    static constexpr bool kTile = (L / 32) <= 64;
    struct Params { float *acc; const UnitInfo *units; int log2N2, log2N, mode; float pf; };
    const Params &p;
    const int tile, unit;
    float rs2;
    __device__ ChiSink(const Params &pp, int tl, int un, int) : p(pp), tile(tl), unit(un), rs2(0.f) {
        if (p.mode == 2) {
            const float rs = p.units[un].rho_scale;
            rs2 = rs * rs;
        }
    }
    __device__ __forceinline__ void update(float *q, float pw) const {
        if (p.mode == 0) *q = pw;
        else if (p.mode == 1) *q += pw;
        else *q = rs2 * fmaf(p.pf, *q, -pw);
    }
    template <int R>
    __device__ __forceinline__ void store(int seq, int b, int stride, const float2 *v) const {
        if constexpr (kTile) {
            chi_park<L, C>(seq, b, stride, v, R);
        } else {
            float *a = p.acc + ((int64_t)unit << p.log2N) + tile * C + seq;
#pragma unroll
            for (int r = 0; r < R; ++r)
                update(a + ((int64_t)(b + r * stride) << p.log2N2), fmaf(v[r].x, v[r].x, v[r].y * v[r].y));
        }
    }
    __device__ __forceinline__ void finish(float2 *) const {
        if constexpr (kTile) {
            __syncthreads();
            float *a = p.acc + ((int64_t)unit << p.log2N) + tile * C;
            // C L elements over C (L / 32) threads: 32 per thread, issued in
            // groups of 8 loads before their read-modify-writes
            constexpr int NT = C * (L / 32);
            constexpr int G = 8;
            static_assert((C * L) % (NT * G) == 0, "tile split");
#pragma unroll 1
            for (int base = 0; base < C * L; base += NT * G) {
                float pw[G], old[G];
                float *q[G];
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int idx = base + g * NT + (int)threadIdx.x;
                    const int seq = idx % C, j1 = idx / C;
                    q[g] = a + seq + ((int64_t)j1 << p.log2N2);
                    pw[g] = chi_tile_row<L, C>(seq)[j1];
                    old[g] = p.mode == 0 ? 0.f : __ldcg(q[g]);
                }
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const float x = p.mode == 0 ? pw[g] : (p.mode == 1 ? old[g] + pw[g] : rs2 * fmaf(p.pf, old[g], -pw[g]));
                    __stcg(q[g], x);
                }
            }
        }
    }
};

// ---------------------------------------------------------------------------
// chi^2 rows kernel (N1 = 1024, N = 2^19 and 2^20).  Pass 1 has written the
// exchange of every sub-band l = 0..p of a batch of nb templates, sub-band l
// of entry b at exch + (l nb + b) N.  Each warp owns one row j2 of one entry
// and transforms it for l = 0..p in turn: the row arrives by a bulk copy
// (cp.async.bulk, mbarrier, bounded wait), stage 0 runs from the staged row,
// and once the last stage has read the warp's region the copy of the same row
// of sub-band l + 1 is issued, so it lands under the arithmetic.  |raw_l|^2 is
// summed in registers over l < p and |raw|^2 (l = p) kept, so
//   chi^2 = rho_scale^2 (p sum_l |raw_l|^2 - |raw|^2)
// is formed without any accumulator in memory.  The CTA's 8 warps own 8
// consecutive rows; they park their 1024 values each in their regions and
// write the 8 x 1024 tile with 8 consecutive samples per 32-byte sector.  The
// sums run in the same order and with the same butterflies as the per-tile
// path, so the results are the same bit for bit.
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ uint32_t cs_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cs_mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cs_addr(bar)) : "memory");
}
__device__ __forceinline__ bool cs_mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(cs_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// generic-proxy accesses of this thread before the async-proxy refill of its region
__device__ __forceinline__ void cs_fence_proxy() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void cs_row_copy(float2 *dst, const float2 *src, uint64_t *bar) {
    constexpr uint32_t bytes = 1024 * sizeof(float2);
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     cs_addr(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     cs_addr(dst)),
                 "l"(src), "r"(bytes), "r"(cs_addr(bar))
                 : "memory");
}

struct ChiWarpSync {
    static __device__ __forceinline__ void sync() { __syncwarp(); }
};

constexpr int kChiWarps = 8;

struct ChiRowsParams {
    const float2 *exch;
    const UnitInfo *full;   // full-band units of the call's template list
    float *chisq;           // [n][N]
    int unit0, nb, p;
    int log2N, log2N2;
    int *status;            // bit 2: a wait ran out
    long long spin_limit;
    int stall;              // test hook: the row copies of list entry `stall` are never issued (-1: none)
};

// last-stage sink: |raw_l|^2 of the thread's 32 outputs (t + 32 q) summed over
// l < p; at l = p (the full band) the sum becomes chi^2 in place; refills the
// region with the next sub-band's row
struct ChiRowAcc {
    float acc[32];
    int l = 0, p = 0;
    float pf = 0.f, rs2 = 0.f;
    float2 *region = nullptr;
    uint64_t *bar = nullptr;
    const float2 *next_src = nullptr;
    __device__ __forceinline__ void after_loads() {
        __syncwarp();
        cs_fence_proxy();
        if (next_src != nullptr && (threadIdx.x & 31) == 0) cs_row_copy(region, next_src, bar);
    }
    template <int R>
    __device__ __forceinline__ void store(int, int, int, const float2 *v) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float pw = fmaf(v[r].x, v[r].x, v[r].y * v[r].y);
            if (l < p) acc[r] = l == 0 ? pw : acc[r] + pw;
            else acc[r] = rs2 * fmaf(pf, acc[r], -pw);
        }
    }
};

__device__ __forceinline__ bool chi_withheld(const ChiRowsParams &p, int64_t r) {
    return p.unit0 + (int)(r >> p.log2N2) == p.stall;
}

__device__ __forceinline__ const float2 *chi_row_src(const ChiRowsParams &p, int64_t r, int l) {
    const int64_t b = r >> p.log2N2, j2 = r & (((int64_t)1 << p.log2N2) - 1);
    if (!MF_DBG(b < p.nb && l <= p.p && ((j2 + 1) << 10) <= ((int64_t)1 << p.log2N), kDbgRows)) return p.exch;
    return p.exch + (((int64_t)l * p.nb + b) << p.log2N) + (j2 << 10);
}

__global__ void __launch_bounds__(kChiWarps * 32, 2) k_chisq_rows(ChiRowsParams p) {
    constexpr int L = 1024;
    using S = FftShape<L>;
    extern __shared__ __align__(16) float2 chi_rows_smem[];
    float2 *tw = chi_rows_smem + kChiWarps * S::STRIDE;
    uint64_t *bars = reinterpret_cast<uint64_t *>(tw + TwTable<L>::SIZE);
    const int w = threadIdx.x >> 5, t = threadIdx.x & 31;
    float2 *region = chi_rows_smem + w * S::STRIDE;
    fill_twiddles<L>(tw);
    if (t == 0) cs_mbar_init(&bars[w]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    // rows of the batch: nb N2, a multiple of 8 (N2 >= 512), so every warp has a row in every round
    const int64_t total = (int64_t)p.nb << p.log2N2;
    const int64_t step = (int64_t)gridDim.x * kChiWarps;
    const float pf = (float)p.p;
    int64_t r0 = (int64_t)blockIdx.x * kChiWarps;
    if (r0 < total && t == 0 && !chi_withheld(p, r0 + w)) cs_row_copy(region, chi_row_src(p, r0 + w, 0), &bars[w]);
    uint32_t parity = 0;
    // a warp whose wait ran out stops waiting and issues no further copies
    // (none of its copies is then in flight), but keeps to the CTA barriers
    bool dead = false;
    for (; r0 < total; r0 += step) {
        const int64_t r = r0 + w;
        ChiRowAcc snk;
        snk.p = p.p;
        snk.pf = pf;
        {
            const float rs = p.full[p.unit0 + (int)(r >> p.log2N2)].rho_scale;
            snk.rs2 = rs * rs;
        }
        snk.region = region;
        snk.bar = &bars[w];
        for (int l = 0; l <= p.p; ++l) {
            // the row of sub-band l has landed (bounded; on expiry the warp is
            // marked dead and the status bit set at the end)
            if (!dead) {
                long long it = 0;
                bool got = true;
                while (!cs_mbar_try_wait(&bars[w], parity)) {
                    if (++it > p.spin_limit) { got = false; break; }
                }
                dead = !__all_sync(0xffffffffu, got);
                parity ^= 1u;
            }
            float2 v[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = region[t + 32 * q];
            Dft<32, +1>::run(v);
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 32; ++q) region[spad(32 * t + q)] = v[q];
            __syncwarp();
            snk.l = l;
            // the next row's first copy waits for the flush
            snk.next_src = (l < p.p && !dead && !chi_withheld(p, r)) ? chi_row_src(p, r, l + 1) : nullptr;
            stockham_stage<L, S::R1, 32, +1, true, ChiRowAcc, ChiWarpSync>(region, tw, 0, t, snk);
        }
        // chi^2 of the row's 1024 samples j2 + N2 (t + 32 q), parked in the warp's region
        float *rowf = reinterpret_cast<float *>(region);
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 32; ++q) rowf[t + 32 * q] = snk.acc[q];
        __syncthreads();
        // the CTA's 8 rows j2 .. j2 + 7 of entry b: 8 consecutive samples per j1
        const int64_t jb = r0 & (((int64_t)1 << p.log2N2) - 1);
        float *out = p.chisq + ((int64_t)(p.unit0 + (r0 >> p.log2N2)) << p.log2N) + jb;
        for (int idx = threadIdx.x; idx < kChiWarps * L; idx += kChiWarps * 32) {
            const int s = idx & (kChiWarps - 1), j1 = idx >> 3;
            __stcs(&out[s + ((int64_t)j1 << p.log2N2)],
                   reinterpret_cast<const float *>(chi_rows_smem + s * S::STRIDE)[j1]);
        }
        cs_fence_proxy();
        __syncthreads();   // the tile is read: the regions may be refilled
        const int64_t rn = r + step;
        if (rn < total && t == 0 && !dead && !chi_withheld(p, rn)) cs_row_copy(region, chi_row_src(p, rn, 0), &bars[w]);
    }
    if (dead && t == 0 && p.status != nullptr) atomicOr(p.status, 2);
}

static size_t chi_rows_smem_bytes() {
    return (size_t)kChiWarps * FftShape<1024>::STRIDE * sizeof(float2) + (size_t)TwTable<1024>::SIZE * sizeof(float2) +
           kChiWarps * sizeof(uint64_t);
}

struct ChiPass2Op {
    const SegDev &seg;
    const UnitInfo *units;
    int unit0, n_units;
    const float2 *exch;
    float *acc;
    int mode;   // 0: first sub-band (store), 1: later sub-band (add), 2: full band (chi^2)
    int p;
    cudaStream_t st;
    template <int N2, int N1>
    cudaError_t run() {
        constexpr int C = seqs_per_cta<N1>(N2);
        const dim3 grid(N2 / C, n_units);
        typename RowSrc<N1, C>::Params sp{exch, seg.log2N1, seg.log2N};
        typename ChiSink<N1, C>::Params kp{acc, units, seg.log2N2, seg.log2N, mode, (float)p};
        return run_pass<N1, C, false, +1, RowSrc<N1, C>, ChiSink<N1, C>>(grid, sp, kp, st, unit0);
    }
};

struct ChiAttrOp {
    template <int N2, int N1>
    cudaError_t run() {
        constexpr int C = seqs_per_cta<N1>(N2);
        return set_pass_attrs<N1, C, false, +1, RowSrc<N1, C>, ChiSink<N1, C>>();
    }
};
}  // namespace

cudaError_t launch_chisq_units(const SegDev &seg, const UnitInfo *all, int n_t, const int32_t *tmpl, int n, int p,
                               UnitInfo *out, int64_t *edges, cudaStream_t st) {
    if (p < 1 || p > kChisqMaxBands) return cudaErrorInvalidValue;
    k_chisq_units<<<n, 128, 0, st>>>(seg, all, n_t, tmpl, n, p, out, edges);
    return cudaGetLastError();
}

cudaError_t launch_chisq_pass2(const SegDev &seg, const UnitInfo *units, int unit0, int n_units, const float2 *exch,
                               float *acc, int mode, int p, cudaStream_t st) {
    ChiPass2Op op{seg, units, unit0, n_units, exch, acc, mode, p, st};
    return dispatch_split(seg.log2N, op);
}

bool chisq_rows_applies(int log2N) { return log2N - log2_n2(log2N) == 10; }

cudaError_t launch_chisq_rows(const SegDev &seg, const float2 *exch, const UnitInfo *full, int unit0, int nb, int p,
                              float *chisq, int *status, long long spin_limit, int stall, int n_sm, cudaStream_t st) {
    if (!chisq_rows_applies(seg.log2N) || nb < 1) return cudaErrorInvalidValue;
    ChiRowsParams q{exch, full, chisq, unit0, nb, p, seg.log2N, seg.log2N2, status, spin_limit, stall};
    const int64_t rounds = ((int64_t)nb << seg.log2N2) / kChiWarps;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(2 * (int64_t)n_sm, rounds));
    k_chisq_rows<<<grid, kChiWarps * 32, chi_rows_smem_bytes(), st>>>(q);
    return cudaGetLastError();
}

MF_DEBUG_READER(dbg_read_chisq)

cudaError_t chisq_kernel_attributes() {
    {
        cudaError_t e0 = init_twiddle_tables();
        if (e0 != cudaSuccess) return e0;
    }
    {
        cudaError_t e1 = cudaFuncSetAttribute(k_chisq_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)chi_rows_smem_bytes());
        if (e1 != cudaSuccess) return e1;
    }
    for (int lg = 10; lg <= 22; ++lg) {
        ChiAttrOp op;
        cudaError_t e = dispatch_split(lg, op);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace mf
