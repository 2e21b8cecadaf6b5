// mf_filter.cu -- the hot path of the bank filter (Eqs. 1, 3, 4 of
// arXiv:0906.4175): per (template, segment) unit
//   k_units    band [k_lo, k_hi) (Sec. 1.1 band rule), sigma from the FP64
//              prefix table, rho and z scale factors, anchor range;
//   k_anchors  the 2PN phase Psi/(2 pi) in FP64 at anchor bins, reduced mod 1,
//              plus its first four k-derivatives (FP32 Taylor coefficients);
//   pass 1     template generation h~_k = e^{-i Psi_k} in registers (FP32
//              quartic Taylor from the nearest anchor, __sincosf of the reduced
//              phase), weighting by W_k = f^(-7/6) conj(s~_k)/S_k, column IFFTs,
//              four-step twiddle, one complex64 exchange write;
//   pass 2     row IFFTs and the rho epilogue: |z|^2 threshold test, argmax with
//              lowest-j tie-break, warp-aggregated trigger append;
//   k_reduce_peaks / k_sort_triggers   deterministic peaks and (tmpl, seg, j)
//              ordered triggers.
// Neither h~(f) nor z(t) is written to memory.
#include "mf_filter.cuh"

namespace mf {

// ---------------------------------------------------------------------------
// per-unit set-up
// ---------------------------------------------------------------------------
// Unit i of a segment is template order[i] (bank order when order is NULL).
__global__ void k_units(SegDev seg, const double *__restrict__ tmpl, int n_t, double f_low, float thr,
                        int log2D, const int *__restrict__ order, UnitInfo *__restrict__ units) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_t) return;
    const int t = order ? order[i] : i;
    const double *T = tmpl + (int64_t)t * kTmplStride;
    const double N = (double)seg.N, fs = seg.fs;
    const double fisco = T[TF_FISCO];
    const double fc = fisco < 0.5 * fs ? fisco : 0.5 * fs;
    int64_t lo = (int64_t)ceil(f_low * N / fs);
    int64_t hi = (int64_t)floor(fc * N / fs) + 1;
    if (lo < 1) lo = 1;
    if (hi > seg.N / 2) hi = seg.N / 2;
    if (hi < lo) hi = lo;
    const double Q = seg.P[hi] - seg.P[lo];              // sum_band f^(-7/3)/S  (Eq. 4 / (4 df A^2))
    const double rs = sqrt(seg.consts->P_tot / Q);
    UnitInfo u;
    u.k_lo = (int32_t)lo;
    u.k_hi = (int32_t)hi;
    u.g_lo = (int32_t)(lo >> log2D);
    u.n_anc = (int32_t)(((hi - 1) >> log2D) - (lo >> log2D) + 1);
    u.rho_scale = (float)rs;
    const double th = (double)thr / rs;
    u.thr2 = (float)(th * th);
    u.z_scale = (float)(4.0 * seg.df * T[TF_AMP] / seg.consts->alpha);
    u.tmpl = t;
    units[i] = u;
}

__global__ void k_anchors(SegDev seg, const double *__restrict__ tmpl, const UnitInfo *__restrict__ units,
                          int unit0, int log2D, int max_anc, float4 *__restrict__ anchors,
                          float *__restrict__ anchors4, int reps) {
    const int b = blockIdx.y;
    const UnitInfo u = units[unit0 + b];
    const double *T = tmpl + (int64_t)u.tmpl * kTmplStride;
    const double c1 = T[TF_C1], c2 = T[TF_C2], c3 = T[TF_C3], c5 = T[TF_C5];
    float4 *out = anchors + (int64_t)b * max_anc;
    float *out4 = anchors4 + (int64_t)b * max_anc;
    const int64_t rep_stride = (int64_t)gridDim.y * max_anc;   // copy k of slot b is slot b + k n_units
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < u.n_anc; i += gridDim.x * blockDim.x) {
        float4 r;
        float r4;
        const int64_t g = (int64_t)u.g_lo + i;
        anchor_record(c1, c2, c3, c5, g, log2D, seg.df, r, r4);
        const int64_t a = anchor_slot_index(g, seg.log2N, seg.log2N1, log2D);
        if (!MF_DBG(a >= 0 && a < max_anc, kDbgAnchor)) continue;
        for (int k = 0; k < reps; ++k) {
            out[a + k * rep_stride] = r;
            out4[a + k * rep_stride] = r4;
        }
    }
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------
MF_DEBUG_READER(dbg_read_filter)

cudaError_t launch_units(const SegDev &seg, const double *tmpl, int n_t, double f_low, float thr, int log2D,
                         const int *order, UnitInfo *units, cudaStream_t st) {
    k_units<<<(n_t + 255) / 256, 256, 0, st>>>(seg, tmpl, n_t, f_low, thr, log2D, order, units);
    return cudaGetLastError();
}

cudaError_t launch_anchors(const SegDev &seg, const double *tmpl, const UnitInfo *units, int unit0, int n_units,
                           int log2D, int max_anc, float4 *anchors, float *anchors4, cudaStream_t st, int reps) {
    if (reps < 1) return cudaErrorInvalidValue;
    const int per = 256;
    int gx = (max_anc + per - 1) / per;
    if (gx > 64) gx = 64;
    k_anchors<<<dim3(gx, n_units), per, 0, st>>>(seg, tmpl, units, unit0, log2D, max_anc, anchors, anchors4, reps);
    return cudaGetLastError();
}

namespace {
struct Pass1Op {
    const SegDev &seg;
    const UnitInfo *units;
    int unit0, n_units, log2D, max_anc, phase_mode;
    const float4 *anchors;
    const float *anchors4;
    float2 *exch;
    const double *tmpl;
    cudaStream_t st;
    template <int N2, int N1>
    cudaError_t run() {
        constexpr int C = seqs_per_cta<N2>(N1);
        typename ExchSink<N2, C, +1, cx_ilog2(N1)>::Params kp{exch, seg.log2N1, seg.log2N};
        const dim3 grid(N1 / C, n_units);
        if (phase_mode == MF_PHASE_FP32) {
            typename TemplateSrcF32<N2, C, cx_ilog2(N1)>::Params sp{seg.W, units, tmpl, (float)seg.df};
            return run_pass<N2, C, true, +1, TemplateSrcF32<N2, C, cx_ilog2(N1)>, ExchSink<N2, C, +1, cx_ilog2(N1)>>(grid, sp, kp, st, unit0);
        }
        typename TemplateSrc<N2, C, cx_ilog2(N1)>::Params sp{seg.W, units, anchors, anchors4, max_anc, log2D};
        return run_pass<N2, C, true, +1, TemplateSrc<N2, C, cx_ilog2(N1)>, ExchSink<N2, C, +1, cx_ilog2(N1)>>(grid, sp, kp, st, unit0);
    }
};

struct Pass2Op {
    const SegDev &seg;
    const UnitInfo *units;
    int unit0, n_units;
    const float2 *exch;
    float4 *partials;
    int seg_idx;
    KeyLayout kl;
    mf_trigger *staged;
    uint64_t *keys;
    unsigned long long *counter;
    int64_t cap;
    cudaStream_t st;
    template <int N2, int N1>
    cudaError_t run() {
        constexpr int C = seqs_per_cta<N1>(N2);
        const int nblk = N2 / C;
        typename RowSrc<N1, C>::Params sp{exch, seg.log2N1, seg.log2N};
        typename RhoSink<N1, C>::Params kp{units, partials, staged, keys, counter, cap,
                                           seg.log2N2, nblk, seg_idx, kl};
        return run_pass<N1, C, false, +1, RowSrc<N1, C>, RhoSink<N1, C>>(dim3(nblk, n_units), sp, kp, st, unit0);
    }
};

struct BlocksOp {
    int nblk = 0;
    template <int N2, int N1>
    cudaError_t run() {
        nblk = N2 / seqs_per_cta<N1>(N2);
        return cudaSuccess;
    }
};

struct AttrOp {
    template <int N2, int N1>
    cudaError_t run() {
        constexpr int C1 = seqs_per_cta<N2>(N1);
        constexpr int C2 = seqs_per_cta<N1>(N2);
        cudaError_t e;
        if ((e = set_pass_attrs<N2, C1, true, +1, TemplateSrc<N2, C1, cx_ilog2(N1)>, ExchSink<N2, C1, +1, cx_ilog2(N1)>>())) return e;
        if ((e = set_pass_attrs<N2, C1, true, +1, TemplateSrcF32<N2, C1, cx_ilog2(N1)>, ExchSink<N2, C1, +1, cx_ilog2(N1)>>())) return e;
        return set_pass_attrs<N1, C2, false, +1, RowSrc<N1, C2>, RhoSink<N1, C2>>();
    }
};
}  // namespace

cudaError_t launch_pass1(const SegDev &seg, const UnitInfo *units, int unit0, int n_units, int log2D, int max_anc,
                         const float4 *anchors, const float *anchors4, float2 *exch, int phase_mode,
                         const double *tmpl, int p1_form, int *status, long long spin_limit, cudaStream_t st,
                         bool narrow) {
    if (p1_form != 1 && pass1_pf_applies(seg.log2N, seg.log2N2, log2D, phase_mode))
        return launch_pass1_pf(seg, units, unit0, n_units, log2D, max_anc, anchors, anchors4, exch, p1_form == 2,
                               status, spin_limit, st, narrow);
    Pass1Op op{seg, units, unit0, n_units, log2D, max_anc, phase_mode, anchors, anchors4, exch, tmpl, st};
    return dispatch_split2(seg.log2N, seg.log2N2, op);
}

cudaError_t launch_pass2(const SegDev &seg, const UnitInfo *units, int unit0, int n_units, const float2 *exch,
                         float4 *partials, int seg_idx, KeyLayout kl, mf_trigger *staged, uint64_t *keys,
                         unsigned long long *counter, int64_t cap, cudaStream_t st) {
    Pass2Op op{seg, units, unit0, n_units, exch, partials, seg_idx, kl, staged, keys, counter, cap, st};
    return dispatch_split2(seg.log2N, seg.log2N2, op);
}

int pass2_blocks(int log2N, int log2N2) {
    BlocksOp op;
    dispatch_split2(log2N, log2N2, op);
    return op.nblk;
}

cudaError_t filter_kernel_attributes() {
    {
        cudaError_t e0 = init_pass_tables();
        if (e0 != cudaSuccess) return e0;
    }
    for (int lg = 10; lg <= 22; ++lg) {
        AttrOp op;
        cudaError_t e = dispatch_split(lg, op);
        if (e == cudaSuccess && alt_log2n2(lg) > 0) e = dispatch_split2(lg, alt_log2n2(lg), op);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// peaks: one warp per unit reduces the pass-2 partials of that unit
// ---------------------------------------------------------------------------
__global__ void k_reduce_peaks(const UnitInfo *__restrict__ units, int n_units, const float4 *__restrict__ partials,
                               int nblk, int seg_idx, int n_seg, mf_peak *__restrict__ peaks) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_units) return;
    float bp = -1.f;
    int bj = 0x7fffffff;
    float bx = 0.f, by = 0.f;
    const float4 *pp = partials + (int64_t)warp * nblk;
    for (int i = lane; i < nblk; i += 32) {
        const float4 c = pp[i];
        const int cj = __float_as_int(c.y);
        if (c.x > bp || (c.x == bp && cj < bj)) { bp = c.x; bj = cj; bx = c.z; by = c.w; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float op = __shfl_xor_sync(0xffffffffu, bp, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        const float ox = __shfl_xor_sync(0xffffffffu, bx, o);
        const float oy = __shfl_xor_sync(0xffffffffu, by, o);
        if (op > bp || (op == bp && oj < bj)) { bp = op; bj = oj; bx = ox; by = oy; }
    }
    if (lane == 0) {
        const UnitInfo u = units[warp];
        mf_peak pk;
        pk.rho = sqrtf(bp) * u.rho_scale;
        pk.j = bj;
        pk.z_re = bx * u.z_scale;
        pk.z_im = by * u.z_scale;
        if (MF_DBG(u.tmpl >= 0 && u.tmpl < n_units && seg_idx < n_seg, kDbgOut))
            peaks[(int64_t)u.tmpl * n_seg + seg_idx] = pk;
    }
}

cudaError_t launch_reduce_peaks(const SegDev &seg, const UnitInfo *units, int n_units, const float4 *partials,
                                int nblk, int seg_idx, int n_seg, mf_peak *peaks, cudaStream_t st) {
    (void)seg;
    const int threads = 256;
    const int blocks = (n_units * 32 + threads - 1) / threads;
    k_reduce_peaks<<<blocks, threads, 0, st>>>(units, n_units, partials, nblk, seg_idx, n_seg, peaks);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Trigger compaction: stable LSD radix sort of the (tmpl, seg, j) keys with
// 8-bit digits over the whole GPU, then a gather into the caller's buffer.
//   k_sort_prepare   n = min(count, cap); *n_out; overflow bit; digit
//                    histograms of every pass over all keys; zeroes the
//                    tile status words and the tile tickets.
//   k_sort_pass      one per digit: CTAs take 2048-key tiles in ticket order,
//                    rank keys stably inside the tile (warp w owns keys
//                    [256 w, 256 w + 256) in 8 rows of 32; __match_any_sync
//                    ranks equal digits of a row in lane order), publish the
//                    tile's digit counts and find the counts of all earlier
//                    tiles by decoupled look-back (Merrill & Garland's
//                    single-pass scan), then scatter.  The last pass writes
//                    the records themselves.
// A tile only waits on tiles with smaller tickets, which running CTAs hold,
// so the look-back always progresses; each wait is still bounded and sets
// status bit 1 when it gives up.
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256, kSortRows = 8, kSortTile = kSortThreads * kSortRows;
constexpr int kSortMaxPass = 8;

__device__ __forceinline__ int64_t sort_count(const unsigned long long *counter, int64_t cap) {
    const unsigned long long total = *counter;
    return (int64_t)(total < (unsigned long long)cap ? total : (unsigned long long)cap);
}

__global__ void __launch_bounds__(kSortThreads)
    k_sort_prepare(const unsigned long long *__restrict__ counter, int64_t cap, int npass,
                   const uint64_t *__restrict__ keys, uint32_t *__restrict__ ghist, uint64_t *__restrict__ tstat,
                   unsigned *__restrict__ tickets, int64_t *__restrict__ n_out, int *status) {
    __shared__ uint32_t h[kSortMaxPass][256];
    const unsigned long long total = *counter;
    const int64_t n = sort_count(counter, cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *n_out = (int64_t)total;
        if (total > (unsigned long long)cap) atomicOr(status, 1);
    }
    if (blockIdx.x == 0 && threadIdx.x < kSortMaxPass) tickets[threadIdx.x] = 0u;
    const int64_t n_tiles = (n + kSortTile - 1) / kSortTile;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = t0; i < n_tiles * 256; i += stride) tstat[i] = 0ull;
    for (int e = threadIdx.x; e < kSortMaxPass * 256; e += blockDim.x) h[e >> 8][e & 255] = 0u;
    __syncthreads();
    for (int64_t i = t0; i < n; i += stride) {
        const uint64_t k = keys[i];
        for (int p = 0; p < npass; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < npass * 256; e += blockDim.x) {
        const uint32_t c = h[e >> 8][e & 255];
        if (c) atomicAdd(&ghist[e], c);
    }
}

// status word of (tile, digit): bits 63..60 = pass + 1, bit 59 = inclusive
// prefix, bit 58 = tile aggregate, bits 31..0 = count
__device__ __forceinline__ uint64_t tstat_load(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void tstat_store(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__global__ void __launch_bounds__(kSortThreads)
    k_sort_pass(const unsigned long long *__restrict__ counter, int64_t cap, int pass, int last,
                const uint64_t *__restrict__ kin, const uint32_t *__restrict__ iin, uint64_t *__restrict__ kout,
                uint32_t *__restrict__ iout, const uint32_t *__restrict__ ghist, uint64_t *tstat,
                unsigned *tickets, const mf_trigger *__restrict__ staged, mf_trigger *__restrict__ out,
                uint32_t *__restrict__ perm_out, int *status, int64_t spin_limit) {
    __shared__ uint32_t whist[kSortThreads / 32][256];
    __shared__ uint32_t base[256];
    __shared__ uint32_t gpre[256];
    __shared__ uint32_t wsum[kSortThreads / 32];
    __shared__ int s_tile, s_abort;
    const int64_t n = sort_count(counter, cap);
    const int64_t n_tiles = (n + kSortTile - 1) / kSortTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, d_own = threadIdx.x;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int shift = 8 * pass;
    const uint64_t tag = (uint64_t)(pass + 1) << 60;
    const uint64_t kPrefix = 1ull << 59, kAgg = 1ull << 58;
    // exclusive prefix of this pass's global digit counts (256 threads = 256 digits)
    {
        const uint32_t x = ghist[pass * 256 + d_own];
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t wo = 0;
        for (int w = 0; w < warp; ++w) wo += wsum[w];
        gpre[d_own] = wo + incl - x;
    }
    if (threadIdx.x == 0) s_abort = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(&tickets[pass], 1u);
        for (int e = lane; e < 256; e += 32) whist[warp][e] = 0u;
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= n_tiles || s_abort) break;
        const int64_t row0 = tile * kSortTile + (int64_t)warp * (32 * kSortRows);
        uint64_t key[kSortRows];
        uint32_t id[kSortRows], dg[kSortRows], lr[kSortRows];
#pragma unroll
        for (int r = 0; r < kSortRows; ++r) {
            const int64_t i = row0 + r * 32 + lane;
            const bool act = i < n;
            key[r] = act ? kin[i] : 0ull;
            id[r] = act ? (iin ? iin[i] : (uint32_t)i) : 0u;
            dg[r] = act ? (uint32_t)((key[r] >> shift) & 255u) : (256u + (uint32_t)lane);
        }
#pragma unroll
        for (int r = 0; r < kSortRows; ++r) {
            const unsigned peers = __match_any_sync(0xffffffffu, dg[r]);
            const uint32_t rank = (uint32_t)__popc(peers & lt_mask);
            const bool act = dg[r] < 256u;
            lr[r] = act ? whist[warp][dg[r]] + rank : 0u;
            __syncwarp();
            if (act && rank == 0) whist[warp][dg[r]] += (uint32_t)__popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // digit d_own: offsets of the warps inside the tile, and the tile total
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) {
            const uint32_t c = whist[w][d_own];
            whist[w][d_own] = tot;
            tot += c;
        }
        uint64_t *my = tstat + tile * 256 + d_own;
        uint32_t excl = 0;
        if (tile == 0) {
            tstat_store(my, tag | kPrefix | tot);
        } else {
            tstat_store(my, tag | kAgg | tot);
            int64_t pt = tile - 1;
            int64_t spins = 0;
            while (pt >= 0) {
                const uint64_t v = tstat_load(tstat + pt * 256 + d_own);
                if ((v >> 60) == (uint64_t)(pass + 1) && (v & (kPrefix | kAgg))) {
                    excl += (uint32_t)v;
                    if (v & kPrefix) break;
                    --pt;
                    continue;
                }
                if (++spins > spin_limit || *(volatile int *)&s_abort) {
                    atomicOr(status, 2);
                    s_abort = 1;
                    break;
                }
                __nanosleep(32);
            }
            tstat_store(my, tag | kPrefix | (uint32_t)(excl + tot));
        }
        base[d_own] = gpre[d_own] + excl;
        __syncthreads();
        if (s_abort) break;
#pragma unroll
        for (int r = 0; r < kSortRows; ++r) {
            if (dg[r] < 256u) {
                const uint32_t pos = base[dg[r]] + whist[warp][dg[r]] + lr[r];
                if (!MF_DBG(pos < (uint64_t)n, kDbgSort)) continue;
                if (last) {
                    out[pos] = staged[id[r]];
                    if (perm_out) perm_out[pos] = id[r];
                } else {
                    kout[pos] = key[r];
                    iout[pos] = id[r];
                }
            }
        }
    }
}

cudaError_t launch_sort_triggers(const unsigned long long *counter, int64_t cap, int key_bits,
                                 const mf_trigger *staged, const uint64_t *keys, uint64_t *keys_tmp,
                                 uint32_t *idx_a, uint32_t *idx_b, uint32_t *ghist, uint64_t *tstat,
                                 unsigned *tickets, mf_trigger *out, uint32_t *perm_out, int64_t *n_out,
                                 int *status, int n_sm, int64_t spin_limit, cudaStream_t st) {
    int npass = key_bits > 0 ? (key_bits + 7) / 8 : 1;
    if (npass > kSortMaxPass) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(ghist, 0, sizeof(uint32_t) * 256 * kSortMaxPass, st);
    if (e != cudaSuccess) return e;
    const int grid = 2 * n_sm;
    k_sort_prepare<<<grid, kSortThreads, 0, st>>>(counter, cap, npass, keys, ghist, tstat, tickets, n_out, status);
    uint64_t *kbuf[2] = {keys_tmp, const_cast<uint64_t *>(keys)};
    uint32_t *ibuf[2] = {idx_a, idx_b};
    const uint64_t *kin = keys;
    const uint32_t *iin = nullptr;
    for (int p = 0; p < npass; ++p) {
        uint64_t *kout = kbuf[p & 1];
        uint32_t *iout = ibuf[p & 1];
        k_sort_pass<<<grid, kSortThreads, 0, st>>>(counter, cap, p, p == npass - 1 ? 1 : 0, kin, iin, kout, iout,
                                                   ghist, tstat, tickets, staged, out, perm_out, status,
                                                   spin_limit);
        kin = kout;
        iin = iout;
    }
    return cudaGetLastError();
}

int sort_launches(int key_bits) { return 1 + (key_bits > 0 ? (key_bits + 7) / 8 : 1); }

}  // namespace mf
