// mf_fused.cu -- the fused persistent bank scheduler: one launch per segment
// runs pass 1 and pass 2 of every (template, segment) unit through a ring of S
// exchange slots small enough to stay in L2.
//
// The grid holds the resident CTAs (two per SM).  The CTAs of a fraction of the
// SMs (the split) are pass-1 workers: they loop over the column tiles of the
// units in order (one atomic
// queue), exactly as the per-batch k_pass1_pf does -- the next tile's W by TMA
// and its anchor rows by bulk copy, issued under the current tile's second
// stage -- and write unit u's exchange into ring slot u % S.  The CTAs of the
// other SMs are pass-2 workers: every warp takes rows from a second atomic queue, exactly as
// k_pass2_rows does (row bulk-copied into the warp's region, the next row's
// copy issued under the current row's last stage, rho epilogue, one partial per
// row).  Dependencies, both on per-unit counters:
//   a row of unit u is copied only once all column tiles of u are written
//     (done1[u] == N1 / C; release by the writing CTA, acquire by the copying lane);
//   a tile of unit u writes its slot only once every row of unit u - S has been
//     copied out of it (done2[u - S] == N2; each row counted when its copy landed).
// Items of each queue start in order and only wait for smaller units, and all
// CTAs are resident, so every wait ends while the GPU makes progress; each is
// still bounded (spin limit with back-off), after which the kernel raises the
// abort flag, sets status bit 1 and every CTA leaves once its own copies in
// flight have landed (again bounded).  Anchors of all units are computed before
// the launch (slot u of the anchor array is unit u).  The arithmetic of every
// tile and row is that of the per-batch kernels, so results are bit-identical.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "mf_pass1.cuh"
#include "mf_rows.cuh"

namespace mf {
namespace {

__device__ __forceinline__ unsigned fz_ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// spin until *ctr >= target; false on abort or when the limit runs out (then
// raises the abort flag and status bit 1)
__device__ bool fz_wait_geq(const unsigned *ctr, unsigned target, unsigned *abort_flag, int *status, long long limit) {
    unsigned ns = 32;
    long long it = 0;
    while (fz_ld_acquire(ctr) < target) {
        if (*(volatile unsigned *)abort_flag) return false;
        if (++it > limit) {
            atomicOr(status, 2);
            atomicExch(abort_flag, 1u);
            return false;
        }
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
    }
    return true;
}

// orders this thread's view of global memory (writes it acquired from other
// threads) before its later async-proxy operations (the bulk copy of a row)
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

struct FusedParams {
    Pass1PfParams p1;      // E = the ring; anchors slot u = unit u; n_items = n_units * tiles
    RowsParams p2;         // exch = the ring; partials [unit][j2]; the stall hook
    unsigned *ctl;         // [0] pass-1 tile head, [1] row head, [2] abort flag (zeroed before launch)
    unsigned *done1;       // per unit: column tiles written
    unsigned *done2;       // per unit: rows copied out of the ring
    int S;                 // ring slots
    int n_p1;              // CTAs [0, n_p1) run pass 1
    float sm_frac;         // > 0: roles by SM instead (see k_filter_fused)
};

// ---------------------------------------------------------------------------
// pass-1 worker (a whole CTA)
// ---------------------------------------------------------------------------
template <int L, int C, int LG1>
__device__ __forceinline__ void fused_p1(const FusedParams &F, const CUtensorMap *wmap, float2 *smem) {
    using S = FftShape<L>;
    constexpr int T = S::T;
    constexpr int NT = C * T;
    constexpr int TILES = (1 << LG1) / C;
    const Pass1PfParams &p = F.p1;
    float2 *wbuf = smem + pass_data_bytes<L, C>() / sizeof(float2);
    float4 *abuf = (float4 *)(wbuf + pf_wbuf_elems<L, C>());
    float *abuf4 = (float *)(abuf + L / 2);
    float2 *tw = (float2 *)(abuf4 + L / 2);
    uint64_t *bar = (uint64_t *)(tw + pf_tw_elems<L>());
    __shared__ int s_next;
    unsigned *abort_flag = F.ctl + 2;
    const int seq = threadIdx.x % C, t = threadIdx.x / C;
    float2 *sq = smem + seq * SeqStride<L, C>::value;
    {
        const float2 *src = g_tw_tables + tw_offset<L>();
        for (int m = threadIdx.x; m < pf_tw_elems<L>(); m += NT) tw[m] = __ldg(&src[m]);
    }
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
        s_next = (int)atomicAdd(&F.ctl[0], 1u);
    }
    __syncthreads();
    const typename ExchSink<L, C, +1, LG1>::Params kp{p.E, LG1, p.log2N};
    const unsigned n2 = 1u << (p.log2N - LG1);   // rows per unit
    int item = s_next;
    uint32_t parity = 0;
    bool in_flight = false;                      // a copy of this CTA has not been waited for
    int pending = -1;                            // unit whose finished tile is released in the next item
    int4 band = make_int4(0, 0, 0, 0);
    __syncthreads();                             // every thread has read s_next
    if (item < p.n_items) {
        band = pf_band(p, item / TILES);
        pf_issue<L, C, LG1, true>(p, wmap, item, band, wbuf, abuf, abuf4, bar);
        in_flight = true;
    }
    while (item < p.n_items) {
        const int u = item / TILES, tile = item - u * TILES;
        const int k_lo = band.x, k_hi = band.y;
        if (threadIdx.x == 0) s_next = (int)atomicAdd(&F.ctl[0], 1u);
        const bool ok = mbar_wait_bounded(bar, parity, p.spin_limit);
        parity ^= 1u;
        in_flight = !ok;
        // inputs staged; the previous tile's last stage has read the column data
        if (__syncthreads_or(!ok || *(volatile unsigned *)abort_flag)) {
            if (threadIdx.x == 0 && !ok) {
                atomicOr(p.status, 2);
                atomicExch(abort_flag, 1u);
            }
            break;
        }
        const int next = s_next;
        const int4 nband = next < p.n_items ? pf_band(p, next / TILES) : make_int4(0, 0, 0, 0);
        pf_stage1<L, C, LG1>(tile, seq, t, k_lo, k_hi, p.log2D, wbuf, abuf, abuf4, sq);
        // release the previous tile: its writes were ordered by the barrier above, and by now (a stage later)
        // they have mostly landed, so the fence waits little; it precedes the slot wait below, so a CTA never
        // waits while holding an unreleased tile
        if (threadIdx.x == 0 && pending >= 0) {
            __threadfence();
            atomicAdd(&F.done1[pending], 1u);
            pending = -1;
        }
        // ring slot u % S is free once every row of unit u - S has been copied out
        bool slot_ok = true;
        if (threadIdx.x == 0 && u >= F.S)
            slot_ok = fz_wait_geq(&F.done2[u - F.S], n2 + (u - F.S == F.p2.stall_unit ? 1u : 0u), abort_flag,
                                  p.status, p.spin_limit);
        // column data complete; every thread has consumed the staged inputs; s_next read
        if (__syncthreads_or(!slot_ok)) break;
        if (next < p.n_items) {
            pf_issue<L, C, LG1, true>(p, wmap, next, nband, wbuf, abuf, abuf4, bar);
            in_flight = true;
        }
        ExchSink<L, C, +1, LG1> snk(kp, tile, u, u % F.S);
        if constexpr (L == 1024) last_stage_1024_split<+1>(sq, tw, seq, t, snk);
        else stockham_stage<L, S::R1, 32, +1, true>(sq, tw, seq, t, snk);
        pending = u;
        item = next;
        band = nband;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (pending >= 0 && !*(volatile unsigned *)abort_flag) {
            __threadfence();
            atomicAdd(&F.done1[pending], 1u);
        }
        if (in_flight) mbar_wait_bounded(bar, parity, p.spin_limit);   // leave no copy landing in freed memory
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// pass-2 worker (each warp on its own; 1024-point rows)
// ---------------------------------------------------------------------------
// Rows are handed out one at a time from an atomic queue (one row at a time
// spreads each unit's rows over the most warps: chunks of four rows left the
// pass-2 warps waiting for units in turn and measured 10 % slower).  Lane 0
// claims a warp's next row at the top of the current one and reads the claim
// after stage 0, so the atomic's latency overlaps the row's first stage.
__device__ __forceinline__ unsigned fz_claim_row(const FusedParams &F) { return atomicAdd(&F.ctl[1], 1u); }

// lane 0: row r's unit has all its column tiles written (false: abort)
__device__ __forceinline__ bool fz_row_ready(const FusedParams &F, unsigned tiles, int64_t total, int &checked,
                                             int64_t r) {
    const RowsParams &p = F.p2;
    if (r >= total) return true;
    const int u = (int)(r >> p.log2N2);
    if (u == checked) return true;
    const unsigned target = tiles + (u == p.stall_unit ? 1u : 0u);   // the test hook never completes
    if (!fz_wait_geq(&F.done1[u], target, F.ctl + 2, p.status, p.spin_limit)) return false;
    fence_proxy_async_global();
    checked = u;
    return true;
}

__device__ __forceinline__ const float2 *fz_row_src(const FusedParams &F, int64_t r) {
    const RowsParams &p = F.p2;
    const int u = (int)(r >> p.log2N2);
    const int64_t j2 = r & (((int64_t)1 << p.log2N2) - 1);
    if (!MF_DBG(u < p.n_units && (j2 + 1) * 1024 <= ((int64_t)1 << p.log2N), kDbgRows)) return p.exch;
    return p.exch + ((int64_t)(u % F.S) << p.log2N) + j2 * 1024;
}

__device__ __forceinline__ void fused_p2(const FusedParams &F, unsigned n_tiles, float2 *smem) {
    constexpr int L = 1024;
    using S = FftShape<L>;
    const RowsParams &p = F.p2;
    const int w = threadIdx.x >> 5, t = threadIdx.x & 31;
    float2 *tw = smem + kWarps * S::STRIDE;
    uint64_t *bars = reinterpret_cast<uint64_t *>(tw + TwTable<L>::SIZE);
    float2 *region = smem + w * S::STRIDE;
    fill_twiddles<L>(tw);
    if (t == 0) mbar_init(&bars[w], 1);
    mbar_fence_init();
    __syncthreads();
    const int64_t total = (int64_t)p.n_units << p.log2N2;
    int checked = -1;
    int64_t r = 0;
    bool ok = true;
    if (t == 0) {
        r = fz_claim_row(F);
        ok = fz_row_ready(F, n_tiles, total, checked, r);
    }
    ok = __shfl_sync(0xffffffffu, (int)ok, 0) != 0;
    r = __shfl_sync(0xffffffffu, r, 0);
    if (!ok) return;
    if (r < total && t == 0) {
        mbar_expect_tx(&bars[w], L * sizeof(float2));
        bulk_copy_g2s(region, fz_row_src(F, r), L * sizeof(float2), &bars[w]);
    }
    bool in_flight = r < total;
    uint32_t parity = 0;
    while (r < total) {
        unsigned claim = 0;
        if (t == 0) claim = fz_claim_row(F);   // read after stage 0
        long long it = 0;
        bool got = true;
        while (!mbar_try_wait(&bars[w], parity)) {
            if (++it > p.spin_limit) { got = false; break; }
        }
        got = __all_sync(0xffffffffu, got);
        if (!got) {
            if (t == 0) {
                atomicOr(p.status, 2);
                atomicExch(F.ctl + 2, 1u);
            }
            return;   // the copy into this warp's region never completed
        }
        parity ^= 1u;
        in_flight = false;
        const int u = (int)(r >> p.log2N2);
        const int j2 = (int)(r & (((int64_t)1 << p.log2N2) - 1));
        if (t == 0) atomicAdd(&F.done2[u], 1u);   // the row has left ring slot u % S
        const UnitInfo uu = p.units[u];
        float2 v[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) v[q] = region[t + 32 * q];
        Dft<32, +1>::run(v);
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 32; ++q) region[spad(32 * t + q)] = v[q];
        __syncwarp();
        // the next row, once its unit is written (its copy is issued in the last stage)
        int64_t rn = 0;
        bool nok = true;
        if (t == 0) {
            rn = claim;
            nok = fz_row_ready(F, n_tiles, total, checked, rn);
        }
        nok = __shfl_sync(0xffffffffu, (int)nok, 0) != 0;
        rn = __shfl_sync(0xffffffffu, rn, 0);
        const bool issue = nok && rn < total;
        GroupRhoSink<L, 1> snk(p, uu, j2, region, &bars[w], issue ? fz_row_src(F, rn) : nullptr);
        stockham_stage<L, S::R1, 32, +1, true, GroupRhoSink<L, 1>, GroupSync<1>>(region, tw, 0, t, snk);
        if (MF_DBG(u < p.n_units && j2 < (1 << p.log2N2), kDbgRows))
            snk.finish(&p.partials[((int64_t)u << p.log2N2) + j2]);
        in_flight = issue;
        if (!nok) break;
        r = rn;
    }
    if (in_flight && t == 0) {   // leave no copy landing in freed memory (bounded)
        long long it = 0;
        while (!mbar_try_wait(&bars[w], parity) && ++it <= p.spin_limit) {
        }
    }
}

template <int L, int C, int LG1>
__global__ void __launch_bounds__(256, 2) k_filter_fused(const FusedParams F, const __grid_constant__ CUtensorMap wmap) {
    extern __shared__ __align__(128) float2 fz_smem[];
    // Roles: by SM (both CTAs of an SM run the same pass, so each SM's instruction cache holds one pass's
    // code; SMs with %smid below the split fraction of %nsmid run pass 1, CTA 0 always pass 1 and the last
    // CTA always pass 2, so each role has a worker), or the first n_p1 CTAs on pass 1.
    bool p1 = (int)blockIdx.x < F.n_p1;
    if (F.sm_frac > 0.f) {
        unsigned smid, nsmid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        asm volatile("mov.u32 %0, %%nsmid;" : "=r"(nsmid));
        p1 = blockIdx.x == 0 || (blockIdx.x + 1 < gridDim.x && (float)smid < F.sm_frac * (float)nsmid);
    }
    if (p1) fused_p1<L, C, LG1>(F, &wmap, fz_smem);
    else fused_p2(F, (unsigned)((1 << LG1) / C), fz_smem);
}

template <int L, int C>
size_t fused_smem() { return std::max<size_t>(pf_smem_bytes<L, C>(), rows_smem<1024>()); }

int g_fused_blocks_per_sm[2] = {0, 0};   // N2 = 512 (N = 2^19), 1024 (N = 2^20)
int g_fused_sms = 0;

struct FusedOp {
    const FusedParams *F;
    const CUtensorMap *wmap;
    cudaStream_t st;
    bool attrs = false;
    template <int N2, int N1>
    cudaError_t run() {
        if constexpr ((N2 == 512 || N2 == 1024) && N1 == 1024) {
            constexpr int C = seqs_per_cta<N2>(N1);
            constexpr int LG1 = cx_ilog2(N1);
            const size_t sm = fused_smem<N2, C>();
            if (attrs) {
                cudaError_t e = cudaFuncSetAttribute(k_filter_fused<N2, C, LG1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)sm);
                if (e != cudaSuccess) return e;
                return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_fused_blocks_per_sm[N2 == 1024 ? 1 : 0],
                                                                     k_filter_fused<N2, C, LG1>, 256, sm);
            }
            const int grid = g_fused_blocks_per_sm[N2 == 1024 ? 1 : 0] * g_fused_sms;
            k_filter_fused<N2, C, LG1><<<grid, 256, sm, st>>>(*F, *wmap);
            return cudaGetLastError();
        } else {
            return cudaErrorNotSupported;
        }
    }
};

}  // namespace

bool fused_applies(int log2N, int log2N2) {
    return (log2N == 19 || log2N == 20) && log2N2 == log2_n2(log2N) && g_fused_sms > 0 &&
           g_fused_blocks_per_sm[log2N == 20 ? 1 : 0] >= 1;
}

int fused_grid(int log2N) { return g_fused_blocks_per_sm[log2N == 20 ? 1 : 0] * g_fused_sms; }

cudaError_t launch_fused(const SegDev &seg, const UnitInfo *units, int n_units, int log2D, int max_anc,
                         const float4 *anchors, const float *anchors4, float2 *ring, int S, double split,
                         unsigned *ctl, unsigned *done1, unsigned *done2, float4 *partials, int seg_idx, KeyLayout kl,
                         mf_trigger *staged, uint64_t *keys, unsigned long long *counter, int64_t cap, int *status,
                         long long spin_limit, int stall_unit, cudaStream_t st) {
    if (!fused_applies(seg.log2N, seg.log2N2) || seg.w_tmap == nullptr || n_units <= 0) return cudaErrorInvalidValue;
    FusedParams F;
    memset(&F, 0, sizeof(F));
    const int C = (8192 >> seg.log2N2) < (1 << seg.log2N1) ? (8192 >> seg.log2N2) : (1 << seg.log2N1);
    F.p1 = Pass1PfParams{seg.W, units, anchors, anchors4, ring, max_anc, log2D, seg.log2N, 0,
                         n_units * ((1 << seg.log2N1) / C), status, spin_limit};
    F.p2.exch = ring;
    F.p2.units = units;
    F.p2.partials = partials;
    F.p2.staged = staged;
    F.p2.keys = keys;
    F.p2.counter = counter;
    F.p2.cap = cap;
    F.p2.unit0 = 0;
    F.p2.n_units = n_units;
    F.p2.log2N = seg.log2N;
    F.p2.log2N2 = seg.log2N2;
    F.p2.seg_idx = seg_idx;
    F.p2.kl = kl;
    F.p2.status = status;
    F.p2.spin_limit = spin_limit;
    F.p2.stall_unit = stall_unit;
    F.ctl = ctl;
    F.done1 = done1;
    F.done2 = done2;
    F.S = S;
    const int grid = fused_grid(seg.log2N);
    F.n_p1 = std::min(grid - 1, std::max(1, (int)(split * grid + 0.5)));
    {   // roles by SM unless MFGB_FUSED_ROLE=cta asks for the first n_p1 CTAs
        const char *e = getenv("MFGB_FUSED_ROLE");
        F.sm_frac = (e && e[0] == 'c') ? 0.f : (float)split;
    }
    FusedOp op{&F, (const CUtensorMap *)seg.w_tmap, st};
    return dispatch_split(seg.log2N, op);
}

cudaError_t fused_kernel_attributes() {
    cudaError_t e = init_pass_tables();   // this translation unit's copies of the Stockham tables and four-step roots
    if (e != cudaSuccess) return e;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_fused_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    for (int lg = 19; lg <= 20; ++lg) {
        FusedOp op{nullptr, nullptr, nullptr, true};
        if ((e = dispatch_split(lg, op)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

MF_DEBUG_READER(dbg_read_fused)

}  // namespace mf
