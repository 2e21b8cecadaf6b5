// mf_persist.cu -- persistent bank scheduler (one launch per segment).
//
// A grid of resident CTAs (two per SM) works through two ordered queues:
//   queue 1, in rounds r = -LA, ..., U-1:  A(r + LA, c) anchor chunks (FP64
//            phase anchors, 1024 per chunk) then P1(r, i) pass-1 tiles
//            (template generation + weighting + column IFFTs);
//   queue 2: P2(u, i) pass-2 tiles (row IFFTs + rho epilogue), unit by unit.
// A CTA starts on queue 1 if (blockIdx mod n_sm) < split, else on queue 2, so
// the two CTAs of an SM usually run the same code; a CTA whose queue is empty
// moves to the other queue.  Items of a queue are handed out in order (one
// atomic head per queue) to running CTAs only.  Dependencies:
//   A(u) needs P1(u - SA) complete (its anchor slot is free),
//   P1(u) needs A(u) complete and P2(u - S) complete (its exchange slot is free),
//   P2(u) needs P1(u) complete.
// Each points to a smaller unit or to an earlier item of the same queue and
// both queues have CTAs from the start, so every wait ends while the GPU makes
// progress; each wait is still bounded (spin limit with __nanosleep back-off),
// after which the kernel raises the abort flag, sets status bit 1
// (MF_ETIMEOUT) and every CTA returns.  Thread 0 decodes the next item and
// reads its counters while the current item runs, and releases each finished
// item during the next one, right after that item's loads are issued, so
// neither the dependency check nor the release fence sits on the critical
// path.  Per-unit peaks are reduced afterwards from the per-tile partials.
#include "mf_filter.cuh"

namespace mf {

constexpr int kItemA = 0, kItemP1 = 1;   // otherwise pass 2

// Device-scope acquire load and release increment (PTX memory model): a
// consumer that observes a counter value with an acquire load, then passes a
// block barrier, sees every write its producer block made before the barrier
// that preceded the producer's release increment.
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned add_release(unsigned *p, unsigned x) {
    unsigned old;
    asm volatile("atom.release.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(x) : "memory");
    return old;
}

// thread 0 only: spin until *ctr >= target; false on abort or timeout
__device__ bool wait_geq(const unsigned *ctr, unsigned target, unsigned *abort_flag, int *status, long long limit) {
    unsigned ns = 32;
    long long it = 0;
    while (ld_acquire(ctr) < target) {
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

// Release: the block barrier orders every thread's prior writes before
// thread 0's device-scope fence (fences are cumulative), which orders them
// before the counter increment that consumers acquire.
__device__ __forceinline__ void block_signal(unsigned *ctr) {
    __syncthreads();
    if (threadIdx.x == 0) add_release(ctr, 1u);
}

// One pass-1 tile: template generation + weighting + column IFFTs -> exchange slot u % S.
template <int N2, int N1>
__device__ __forceinline__ void persist_p1(float2 *smem, const float2 *tw, void *scratch,
                                        const typename TemplateSrc<N2, seqs_per_cta<N2>(N1), cx_ilog2(N1)>::Params &sp,
                                        const typename ExchSink<N2, seqs_per_cta<N2>(N1), +1, cx_ilog2(N1)>::Params &kp, int u,
                                        int tile, int S, int SA, unsigned *&pending) {
    constexpr int C1 = seqs_per_cta<N2>(N1);
    TemplateSrc<N2, C1, cx_ilog2(N1)> src(sp, tile, u, u % SA, scratch);
    src.rel = pending;
    pending = nullptr;
    ExchSink<N2, C1, +1, cx_ilog2(N1)> snk(kp, tile, u, u % S);
    cta_fft<N2, C1, true, +1>(smem, tw, src, snk);
}

// One pass-2 tile: row IFFTs of exchange slot u % S + rho epilogue -> partials[u][tile].
template <int N2, int N1>
__device__ __forceinline__ void persist_p2(float2 *smem, const float2 *tw,
                                        const typename RowSrc<N1, seqs_per_cta<N1>(N2)>::Params &sp,
                                        const typename RhoSink<N1, seqs_per_cta<N1>(N2)>::Params &kp, int u, int tile,
                                        int S, unsigned *&pending) {
    constexpr int C2 = seqs_per_cta<N1>(N2);
    RowSrc<N1, C2> src(sp, tile, u, u % S, nullptr);
    src.rel = pending;
    pending = nullptr;
    RhoSink<N1, C2> snk(kp, tile, u, 0);
    cta_fft<N1, C2, false, +1>(smem, tw, src, snk);
    snk.finish(smem);
}

// One anchor chunk of unit u: records [tile * 1024, tile * 1024 + 1024) into slot u % SA.
__device__ __noinline__ void persist_anchors(const PersistParams &P, int u, int tile) {
    const UnitInfo ui = P.units[u];
    const double *T = P.tmpl + (int64_t)ui.tmpl * kTmplStride;
    const double c1 = T[TF_C1], c2 = T[TF_C2], c3 = T[TF_C3], c5 = T[TF_C5];
    float4 *out = P.anchors + (int64_t)(u % P.SA) * P.max_anc;
    float *out4 = P.anchors4 + (int64_t)(u % P.SA) * P.max_anc;
    const int lo = tile * 1024, hi = min(ui.n_anc, lo + 1024);
    for (int i = lo + (int)threadIdx.x; i < hi; i += 256) {
        float4 r;
        float r4;
        const int64_t g = (int64_t)ui.g_lo + i;
        anchor_record(c1, c2, c3, c5, g, P.log2D, P.seg.df, r, r4);
        const int64_t a = anchor_slot_index(g, P.seg.log2N, P.seg.log2N1, P.log2D);
        if (!MF_DBG(a >= 0 && a < P.max_anc, kDbgAnchor)) continue;
        out[a] = r;
        out4[a] = r4;
    }
}

struct ItemDesc {
    int u, phase, tile;
};

__device__ __forceinline__ ItemDesc decode_item(const PersistParams &P, int qid, int q, int n1, int n2) {
    if (qid == 2) return ItemDesc{q / n2, 2, q % n2};
    for (int i = 0; i < P.n_reg; ++i) {
        const QueueRegime &g = P.reg[i];
        const int end = g.first + g.size * g.rounds;
        if (q >= end) continue;
        const int rel = q - g.first;
        const int rr = rel / g.size;
        int pos = rel - rr * g.size;
        const int rho = g.rho0 + rr;
        if (g.flags & 1) {
            if (pos < P.nA) return ItemDesc{rho + P.LA, kItemA, pos};
            pos -= P.nA;
        }
        return ItemDesc{rho, kItemP1, pos};
    }
    return ItemDesc{0, kItemP1, 0};
}

// Counters (address, target) that must be reached before item d may run.
struct Deps {
    const unsigned *c0, *c1;
    unsigned t0, t1;
};

__device__ __forceinline__ Deps item_deps(const PersistParams &P, const ItemDesc &d, int n1, int n2) {
    Deps r{nullptr, nullptr, 0u, 0u};
    if (d.phase == kItemA) {
        if (d.u >= P.SA) { r.c0 = P.done1 + (d.u - P.SA); r.t0 = (unsigned)n1; }
    } else if (d.phase == kItemP1) {
        r.c0 = P.doneA + d.u;
        r.t0 = (unsigned)P.nA;
        if (d.u >= P.S) { r.c1 = P.done2 + (d.u - P.S); r.t1 = (unsigned)n2; }
    } else {
        r.c0 = P.done1 + d.u;
        r.t0 = (unsigned)n1 + (d.u == P.stall_unit ? 1u : 0u);
    }
    return r;
}

__device__ __forceinline__ unsigned *item_counter(const PersistParams &P, int phase, int u) {
    return (phase == kItemA ? P.doneA : (phase == kItemP1 ? P.done1 : P.done2)) + u;
}

// thread 0: release a deferred counter now (see release_hook)
__device__ __forceinline__ void flush_release(unsigned *&pending) {
    if (pending) {
        __threadfence();
        atomicAdd(pending, 1u);
        pending = nullptr;
    }
}

template <int N2, int N1>
__global__ void __launch_bounds__(256, 2)
    k_filter_persistent(PersistParams P, typename TemplateSrc<N2, seqs_per_cta<N2>(N1), cx_ilog2(N1)>::Params sp1,
                        typename ExchSink<N2, seqs_per_cta<N2>(N1), +1, cx_ilog2(N1)>::Params kp1,
                        typename RowSrc<N1, seqs_per_cta<N1>(N2)>::Params sp2,
                        typename RhoSink<N1, seqs_per_cta<N1>(N2)>::Params kp2) {
    constexpr int C1 = seqs_per_cta<N2>(N1);
    constexpr int C2 = seqs_per_cta<N1>(N2);
    static_assert(C1 * (N2 / 32) == 256 && C2 * (N1 / 32) == 256, "persistent path needs 256-thread tiles");
    constexpr int n1 = N1 / C1;
    constexpr int n2 = N2 / C2;
    extern __shared__ float2 smem[];
    unsigned *abort_flag = P.ctl + 1;
    constexpr size_t d1 = pass_data_bytes<N2, C1>(), d2 = pass_data_bytes<N1, C2>();
    float2 *tw1 = smem + (d1 > d2 ? d1 : d2) / sizeof(float2);
    float2 *tw2 = tw1 + TwTable<N2>::SIZE;
    void *scratch1 = tw2 + TwTable<N1>::SIZE;
    fill_twiddles<N2>(tw1);
    fill_twiddles<N1>(tw2);
    // Item pipeline (per queue).  s_desc[par] is the item this block runs now;
    // while it runs, thread 0 decodes the next item (index qn, reserved one
    // item earlier), reads its counters and reserves the index after it.  At
    // the end thread 0 publishes the next descriptor and one barrier follows.
    // If the counters read ahead do not show the next item's dependencies
    // (rare) it is published as pending (state 2): thread 0 then releases its
    // deferred counter (the dependency may be this block's own item), waits,
    // and a second barrier publishes the outcome.
    __shared__ int4 s_desc[2];   // {unit, phase, tile, state}: state 0 stop, 1 run, 2 pending
    __shared__ int4 s_nd;        // thread 0's decoded next item
    __shared__ Deps s_dep;       // and its dependencies
    __shared__ int s_next_ok;
    unsigned *pending = nullptr;   // thread 0: finished item whose counter is not yet released
    bool aborted = false;
    const int role = ((int)(blockIdx.x % (unsigned)P.n_sm) < P.split) ? 1 : 2;
    for (int pass = 0; pass < 2 && !aborted; ++pass) {
        const int qid = pass == 0 ? role : 3 - role;
        unsigned *head = qid == 1 ? P.ctl : P.ctl + 2;
        const int nq = qid == 1 ? P.n_items1 : P.n_items2;
        int qn = 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            const int q0 = (int)atomicAdd(head, 1u);
            int4 d = make_int4(0, 0, 0, 0);
            if (q0 < nq && !*(volatile unsigned *)abort_flag) {
                const ItemDesc it0 = decode_item(P, qid, q0, n1, n2);
                const Deps dp = item_deps(P, it0, n1, n2);
                flush_release(pending);
                bool ok = true;
                if (dp.c0) ok = wait_geq(dp.c0, dp.t0, abort_flag, P.status, P.spin_limit);
                if (ok && dp.c1) ok = wait_geq(dp.c1, dp.t1, abort_flag, P.status, P.spin_limit);
                d = make_int4(it0.u, it0.phase, it0.tile, ok ? 1 : 0);
            }
            s_desc[0] = d;
            qn = (int)atomicAdd(head, 1u);
        }
        __syncthreads();
        int par = 0;
        for (;;) {
            const int4 d = s_desc[par];
            if (d.w == 0) {
                aborted = *(volatile unsigned *)abort_flag != 0u;
                break;
            }
            const int u = d.x, phase = d.y, tile = d.z;
            if (!MF_DBG(u >= 0 && (int64_t)u * n2 < P.n_items2 &&
                            tile >= 0 && tile < (phase == kItemA ? P.nA : (phase == kItemP1 ? n1 : n2)),
                        kDbgQueue)) {
                aborted = true;   // a decoding error: stop the block (the debug word reports it)
                break;
            }
            // look-ahead (thread 0)
            unsigned nv0 = 0u, nv1 = 0u, nab = 0u;
            int qn2 = 0;
            if (threadIdx.x == 0) {
                s_next_ok = qn < nq;
                if (s_next_ok) {
                    const ItemDesc nd = decode_item(P, qid, qn, n1, n2);
                    const Deps dp = item_deps(P, nd, n1, n2);
                    s_nd = make_int4(nd.u, nd.phase, nd.tile, 0);
                    s_dep = dp;
                    nv0 = dp.c0 ? ld_acquire(dp.c0) : 0u;
                    nv1 = dp.c1 ? ld_acquire(dp.c1) : 0u;
                }
                nab = *(volatile unsigned *)abort_flag;
                qn2 = (int)atomicAdd(head, 1u);
            }
            if (phase == kItemA) {
                if (threadIdx.x == 0) flush_release(pending);
                persist_anchors(P, u, tile);
            } else if (phase == kItemP1) {
                persist_p1<N2, N1>(smem, tw1, scratch1, sp1, kp1, u, tile, P.S, P.SA, pending);
            } else {
                persist_p2<N2, N1>(smem, tw2, sp2, kp2, u, tile, P.S, pending);
            }
            if (threadIdx.x == 0) {
                pending = item_counter(P, phase, u);   // released during the next item
                int4 e = make_int4(0, 0, 0, 0);
                if (s_next_ok && !nab) {
                    const Deps dp = s_dep;
                    const bool sat = (!dp.c0 || nv0 >= dp.t0) && (!dp.c1 || nv1 >= dp.t1);
                    e = s_nd;
                    e.w = sat ? 1 : 2;
                    if (P.stats) {
                        atomicAdd(P.stats + 4 * e.y + 2, 1ull);
                        if (!sat) atomicAdd(P.stats + 4 * e.y + 3, 1ull);
                    }
                }
                s_desc[par ^ 1] = e;
                qn = qn2;
            }
            __syncthreads();   // publishes the next descriptor; this item's writes are issued
            par ^= 1;
            if (s_desc[par].w == 2) {
                if (threadIdx.x == 0) {
                    const long long t0 = clock64();
                    flush_release(pending);
                    const Deps dp = s_dep;
                    bool ok = true;
                    if (dp.c0 && nv0 < dp.t0) ok = wait_geq(dp.c0, dp.t0, abort_flag, P.status, P.spin_limit);
                    if (ok && dp.c1 && nv1 < dp.t1) ok = wait_geq(dp.c1, dp.t1, abort_flag, P.status, P.spin_limit);
                    if (P.stats) atomicAdd(P.stats + 4 * s_desc[par].y + 1, (unsigned long long)(clock64() - t0));
                    s_desc[par].w = ok ? 1 : 0;
                }
                __syncthreads();
            }
        }
    }
    if (threadIdx.x == 0) flush_release(pending);
    (void)C2;
}

template <int N2, int N1>
size_t persist_smem() {
    constexpr int C1 = seqs_per_cta<N2>(N1);
    constexpr int C2 = seqs_per_cta<N1>(N2);
    const size_t a = pass_data_bytes<N2, C1>(), b = pass_data_bytes<N1, C2>();
    return (a > b ? a : b) + sizeof(float2) * (TwTable<N2>::SIZE + TwTable<N1>::SIZE) +
           TemplateSrc<N2, C1, cx_ilog2(N1)>::kScratchBytes;
}

namespace {
struct PersistOp {
    const PersistParams &P;
    int grid;
    cudaStream_t st;
    template <int N2, int N1>
    cudaError_t run() {
        if constexpr (N2 * N1 < 8192) {
            return cudaErrorInvalidValue;
        } else {
            constexpr int C1 = seqs_per_cta<N2>(N1);
            constexpr int C2 = seqs_per_cta<N1>(N2);
            typename TemplateSrc<N2, C1, cx_ilog2(N1)>::Params sp1{P.seg.W, P.units, P.anchors, P.anchors4, P.max_anc,
                                                                   P.log2D};
            typename ExchSink<N2, C1, +1, cx_ilog2(N1)>::Params kp1{P.exch, P.seg.log2N1, P.seg.log2N};
            typename RowSrc<N1, C2>::Params sp2{P.exch, P.seg.log2N1, P.seg.log2N};
            typename RhoSink<N1, C2>::Params kp2{P.units, P.partials, P.staged, P.keys, P.counter, P.cap,
                                                 P.seg.log2N2, N2 / C2, P.seg_idx, P.kl};
            k_filter_persistent<N2, N1><<<grid, 256, persist_smem<N2, N1>(), st>>>(P, sp1, kp1, sp2, kp2);
            return cudaGetLastError();
        }
    }
};
struct PersistAttrOp {
    int log2N;
    int *blocks_per_sm;
    template <int N2, int N1>
    cudaError_t run() {
        if constexpr (N2 * N1 < 8192) {
            return cudaSuccess;
        } else {
            cudaError_t e = cudaFuncSetAttribute(k_filter_persistent<N2, N1>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)persist_smem<N2, N1>());
            if (e != cudaSuccess) return e;
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm + log2N, k_filter_persistent<N2, N1>,
                                                                 256, persist_smem<N2, N1>());
        }
    }
};
struct TilesOp {
    int n1 = 0, n2 = 0;
    template <int N2, int N1>
    cudaError_t run() {
        n1 = N1 / seqs_per_cta<N2>(N1);
        n2 = N2 / seqs_per_cta<N1>(N2);
        return cudaSuccess;
    }
};
int g_blocks_per_sm[32];
}  // namespace

MF_DEBUG_READER(dbg_read_persist)

cudaError_t persist_kernel_attributes() {
    {
        cudaError_t e0 = init_pass_tables();
        if (e0 != cudaSuccess) return e0;
    }
    for (int lg = 13; lg <= 22; ++lg) {
        PersistAttrOp op{lg, g_blocks_per_sm};
        cudaError_t e = dispatch_split(lg, op);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int persist_blocks_per_sm(int log2N) { return (log2N >= 13 && log2N <= 22) ? g_blocks_per_sm[log2N] : 0; }

void persist_tiles(int log2N, int *n1, int *n2) {
    TilesOp op;
    dispatch_split(log2N, op);
    *n1 = op.n1;
    *n2 = op.n2;
}

cudaError_t launch_persistent(const PersistParams &P, int grid, cudaStream_t st) {
    PersistOp op{P, grid, st};
    return dispatch_split(P.seg.log2N, op);
}

}  // namespace mf
