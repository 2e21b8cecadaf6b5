// mf_persist.cu -- persistent bank scheduler (one launch per segment).
//
// A grid of resident CTAs takes work items from an ordered queue (one atomic
// counter; each CTA reserves its next item while it works on the current
// one).  For unit u (a template on this segment) the items are
//   A(u, c)   anchors chunk c (FP64 phase anchors, 1024 per chunk)
//   P1(u, i)  pass-1 tile i: template generation + weighting + column IFFTs
//   P2(u, i)  pass-2 tile i: row IFFTs + rho epilogue
// interleaved in rounds r = 0, 1, ...:  A(r + LA), P1(r), P2(r - D2), so that
// anchor work (FP64), column FFTs and row FFTs of different templates run side
// by side.  Exchange buffers form a ring of S slots and anchor tables a ring
// of SA slots.  Every dependency points to an item earlier in the queue and
// items are handed out in queue order to running CTAs only, so the earliest
// unfinished item can always run and every wait ends as long as the GPU makes
// progress; each wait is still bounded (spin limit with __nanosleep back-off),
// after which the kernel raises the abort flag, sets status bit 1
// (MF_ETIMEOUT) and every CTA returns.  Items are decoded arithmetically from
// the round structure, and thread 0 reads the next item's dependency counters
// before the current item's release barrier, so a satisfied dependency costs
// no memory round trip on the critical path.
//   P1(u) waits for A(u) complete and for P2(u - S) complete (slot free);
//   A(u) waits for P1(u - SA) complete (anchor slot free);
//   P2(u) waits for P1(u) complete.
// The last P2 tile of a unit reduces the unit's per-tile partial argmaxes into
// its peak record.
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
                                        const typename TemplateSrc<N2, seqs_per_cta<N2>(N1)>::Params &sp,
                                        const typename ExchSink<N2, seqs_per_cta<N2>(N1), +1>::Params &kp, int u,
                                        int tile, int S, int SA) {
    constexpr int C1 = seqs_per_cta<N2>(N1);
    TemplateSrc<N2, C1> src(sp, tile, u, u % SA, scratch);
    ExchSink<N2, C1, +1> snk(kp, tile, u, u % S);
    cta_fft<N2, C1, true, +1>(smem, tw, src, snk);
}

// One pass-2 tile: row IFFTs of exchange slot u % S + rho epilogue -> partials[u][tile].
template <int N2, int N1>
__device__ __forceinline__ void persist_p2(float2 *smem, const float2 *tw,
                                        const typename RowSrc<N1, seqs_per_cta<N1>(N2)>::Params &sp,
                                        const typename RhoSink<N1, seqs_per_cta<N1>(N2)>::Params &kp, int u, int tile,
                                        int S) {
    constexpr int C2 = seqs_per_cta<N1>(N2);
    RowSrc<N1, C2> src(sp, tile, u, u % S, nullptr);
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
        anchor_record(c1, c2, c3, c5, (int64_t)ui.g_lo + i, P.log2D, P.seg.df, r, r4);
        out[i] = r;
        out4[i] = r4;
    }
}

// The last pass-2 tile of unit u reduces the unit's partial argmaxes (warp 0).
template <int N2, int N1>
__device__ __noinline__ void persist_peak(const PersistParams &P, int u) {
    constexpr int n2 = N2 / seqs_per_cta<N1>(N2);
    __threadfence();   // the other tiles' partials were released before their increments
    const int lane = threadIdx.x;
    float bp = -1.f, bx = 0.f, by = 0.f;
    int bj = 0x7fffffff;
    const float4 *pp = P.partials + (int64_t)u * n2;
    for (int i = lane; i < n2; i += 32) {
        const float4 c = __ldcg(&pp[i]);
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
        const UnitInfo ui = P.units[u];
        mf_peak pk;
        pk.rho = sqrtf(bp) * ui.rho_scale;
        pk.j = bj;
        pk.z_re = bx * ui.z_scale;
        pk.z_im = by * ui.z_scale;
        P.peaks[(int64_t)ui.tmpl * P.n_seg + P.seg_idx] = pk;
    }
}

struct ItemDesc {
    int u, phase, tile;
};

__device__ __forceinline__ ItemDesc decode_item(const PersistParams &P, int q, int n1) {
    ItemDesc d{0, 2, 0};
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
        if (g.flags & 2) {
            if (pos < n1) return ItemDesc{rho, kItemP1, pos};
            pos -= n1;
        }
        return ItemDesc{rho - P.D2, 2, pos};
    }
    return d;
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

template <int N2, int N1>
__global__ void __launch_bounds__(256, 2)
    k_filter_persistent(PersistParams P, typename TemplateSrc<N2, seqs_per_cta<N2>(N1)>::Params sp1,
                        typename ExchSink<N2, seqs_per_cta<N2>(N1), +1>::Params kp1,
                        typename RowSrc<N1, seqs_per_cta<N1>(N2)>::Params sp2,
                        typename RhoSink<N1, seqs_per_cta<N1>(N2)>::Params kp2) {
    constexpr int C1 = seqs_per_cta<N2>(N1);
    constexpr int C2 = seqs_per_cta<N1>(N2);
    static_assert(C1 * (N2 / 32) == 256 && C2 * (N1 / 32) == 256, "persistent path needs 256-thread tiles");
    constexpr int n1 = N1 / C1;
    constexpr int n2 = N2 / C2;
    extern __shared__ float2 smem[];
    unsigned *abort_flag = P.ctl + 1;   // P.ctl[0] is the queue head
    constexpr size_t d1 = pass_data_bytes<N2, C1>(), d2 = pass_data_bytes<N1, C2>();
    float2 *tw1 = smem + (d1 > d2 ? d1 : d2) / sizeof(float2);
    float2 *tw2 = tw1 + TwTable<N2>::SIZE;
    void *scratch1 = tw2 + TwTable<N1>::SIZE;
    fill_twiddles<N2>(tw1);
    fill_twiddles<N1>(tw2);
    unsigned *head = P.ctl;
    // Item pipeline.  s_desc[par] is the item this block runs now; while it
    // runs, thread 0 decodes the next item (index qn, reserved one item
    // earlier) and reads its dependency counters, and reserves the index after
    // it.  At the end thread 0 publishes the next descriptor, one barrier
    // follows, and only then does thread 0 release the finished item, so the
    // other warps start the next item while the release (which waits for this
    // item's stores) is in flight.  If the counters read ahead do not yet show
    // the next item's dependencies (rare), the descriptor is published as
    // "pending": thread 0 releases first (the dependency may be this block's
    // own item), then waits, then a second barrier publishes the outcome.
    __shared__ int4 s_desc[2];   // {unit, phase, tile, state}: state 0 stop, 1 run, 2 pending
    __shared__ int4 s_nd;        // thread 0's decoded next item
    __shared__ Deps s_dep;       // and its dependencies
    __shared__ int s_next_ok;
    int qn = 0;
    if (threadIdx.x == 0) {
        const int q0 = (int)atomicAdd(head, 1u);
        int4 d = make_int4(0, 0, 0, 0);
        if (q0 < P.n_items) {
            const ItemDesc it0 = decode_item(P, q0, n1);
            const Deps dp = item_deps(P, it0, n1, n2);
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
        if (d.w == 0) break;
        const int u = d.x, phase = d.y, tile = d.z;
        // look-ahead (thread 0): decode the next item into shared memory, read
        // its counters (the values stay in registers), reserve the index after it
        unsigned nv0 = 0u, nv1 = 0u, nab = 0u;
        int qn2 = 0;
        if (threadIdx.x == 0) {
            s_next_ok = qn < P.n_items;
            if (s_next_ok) {
                const ItemDesc nd = decode_item(P, qn, n1);
                const Deps dp = item_deps(P, nd, n1, n2);
                s_nd = make_int4(nd.u, nd.phase, nd.tile, 0);
                s_dep = dp;
                nv0 = dp.c0 ? ld_acquire(dp.c0) : 0u;
                nv1 = dp.c1 ? ld_acquire(dp.c1) : 0u;
            }
            nab = *(volatile unsigned *)abort_flag;
            qn2 = (int)atomicAdd(head, 1u);
        }
        unsigned *done_ctr;
        if (phase == kItemA) {
            persist_anchors(P, u, tile);
            done_ctr = P.doneA + u;
        } else if (phase == kItemP1) {
            persist_p1<N2, N1>(smem, tw1, scratch1, sp1, kp1, u, tile, P.S, P.SA);
            done_ctr = P.done1 + u;
        } else {
            persist_p2<N2, N1>(smem, tw2, sp2, kp2, u, tile, P.S);
            done_ctr = P.done2 + u;
        }
        if (threadIdx.x == 0) {
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
        unsigned old = 0u;
        if (threadIdx.x == 0) old = add_release(done_ctr, 1u);
        if (phase != kItemA && phase != kItemP1 && threadIdx.x < 32) {
            old = __shfl_sync(0xffffffffu, old, 0);
            if (old == (unsigned)(n2 - 1)) persist_peak<N2, N1>(P, u);
        }
        par ^= 1;
        if (s_desc[par].w == 2) {
            if (threadIdx.x == 0) {
                const long long t0 = clock64();
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
    (void)C2;
}

template <int N2, int N1>
size_t persist_smem() {
    constexpr int C1 = seqs_per_cta<N2>(N1);
    constexpr int C2 = seqs_per_cta<N1>(N2);
    const size_t a = pass_data_bytes<N2, C1>(), b = pass_data_bytes<N1, C2>();
    return (a > b ? a : b) + sizeof(float2) * (TwTable<N2>::SIZE + TwTable<N1>::SIZE) +
           TemplateSrc<N2, C1>::kScratchBytes;
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
            typename TemplateSrc<N2, C1>::Params sp1{P.seg.W, P.units, P.anchors, P.anchors4, P.max_anc,
                                                     P.seg.log2N1, P.log2D};
            typename ExchSink<N2, C1, +1>::Params kp1{P.exch, P.seg.log2N1, P.seg.log2N};
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

cudaError_t persist_kernel_attributes() {
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
