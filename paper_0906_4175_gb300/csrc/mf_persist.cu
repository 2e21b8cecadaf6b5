// mf_persist.cu -- persistent bank scheduler (one launch per segment).
//
// A fixed grid (resident CTAs) pulls work items from an ordered queue built on
// the host.  For unit u (a template on this segment) the items are
//   A(u, c)   anchors chunk c (FP64 phase anchors, 1024 per chunk)
//   P1(u, i)  pass-1 tile i: template generation + weighting + column IFFTs
//   P2(u, i)  pass-2 tile i: row IFFTs + rho epilogue
// interleaved in rounds r = 0, 1, ...:  A(r + LA), P1(r), P2(r - D2), so that
// anchor work (FP64), column FFTs and row FFTs of different templates run side
// by side.  Exchange buffers form a ring of S slots and anchor tables a ring
// of SA slots.  Every dependency points to an item earlier in the queue, and
// items are taken in queue order by running CTAs, so every wait ends as long
// as the GPU makes progress; each wait is still bounded (spin limit with
// __nanosleep back-off), after which the kernel raises the abort flag, sets
// status bit 1 (MF_ETIMEOUT) and every CTA returns.
//   P1(u) waits for A(u) complete and for P2(u - S) complete (slot free);
//   A(u) waits for P1(u - SA) complete (anchor slot free);
//   P2(u) waits for P1(u) complete.
// The last P2 tile of a unit reduces the unit's per-tile partial argmaxes into
// its peak record.
#include "mf_filter.cuh"

namespace mf {

constexpr int kItemA = 0, kItemP1 = 1, kItemP2 = 2;

// thread 0 only: spin until *ctr >= target; false on abort or timeout
__device__ bool wait_geq(const unsigned *ctr, unsigned target, unsigned *abort_flag, int *status, long long limit) {
    unsigned ns = 32;
    long long it = 0;
    while (*(volatile const unsigned *)ctr < target) {
        if (*(volatile unsigned *)abort_flag) return false;
        if (++it > limit) {
            atomicOr(status, 2);
            atomicExch(abort_flag, 1u);
            return false;
        }
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
    }
    __threadfence();
    return true;
}

// All threads: thread 0 waits, the block learns the outcome.
__device__ __forceinline__ bool block_wait(const unsigned *ctr, unsigned target, unsigned *abort_flag, int *status,
                                           int *s_flag, long long limit) {
    if (threadIdx.x == 0) *s_flag = wait_geq(ctr, target, abort_flag, status, limit) ? 1 : 0;
    __syncthreads();
    const bool ok = *s_flag != 0;
    __syncthreads();
    return ok;
}

// Release: the block barrier orders every thread's prior writes before
// thread 0's device-scope fence (fences are cumulative), which orders them
// before the counter increment that consumers acquire.
__device__ __forceinline__ void block_signal(unsigned *ctr) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
    }
}

// One pass-1 tile: template generation + weighting + column IFFTs -> exchange slot u % S.
template <int N2, int N1>
__device__ __noinline__ void persist_p1(float2 *smem, const typename TemplateSrc<N2, seqs_per_cta<N2>(N1)>::Params &sp,
                                        const typename ExchSink<N2, seqs_per_cta<N2>(N1), +1>::Params &kp, int u,
                                        int tile, int S, int SA) {
    constexpr int C1 = seqs_per_cta<N2>(N1);
    TemplateSrc<N2, C1> src(sp, tile, u, u % SA);
    ExchSink<N2, C1, +1> snk(kp, tile, u, u % S);
    cta_fft<N2, C1, true, +1>(smem, src, snk);
}

// One pass-2 tile: row IFFTs of exchange slot u % S + rho epilogue -> partials[u][tile].
template <int N2, int N1>
__device__ __noinline__ void persist_p2(float2 *smem, const typename RowSrc<N1, seqs_per_cta<N1>(N2)>::Params &sp,
                                        const typename RhoSink<N1, seqs_per_cta<N1>(N2)>::Params &kp, int u, int tile,
                                        int S) {
    constexpr int C2 = seqs_per_cta<N1>(N2);
    RowSrc<N1, C2> src(sp, tile, u, u % S);
    RhoSink<N1, C2> snk(kp, tile, u, 0);
    cta_fft<N1, C2, false, +1>(smem, src, snk);
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
    __threadfence();
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
    __shared__ int s_item, s_flag;
    __shared__ unsigned s_old;
    unsigned *head = P.ctl, *abort_flag = P.ctl + 1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (*(volatile unsigned *)abort_flag) ? P.n_items : (int)atomicAdd(head, 1u);
        __syncthreads();
        const int q = s_item;
        if (q >= P.n_items) break;
        const int2 it = P.items[q];
        const int u = it.x, phase = it.y >> 16, tile = it.y & 0xffff;
        if (phase == kItemA) {
            if (u >= P.SA && !block_wait(P.done1 + (u - P.SA), n1, abort_flag, P.status, &s_flag, P.spin_limit))
                break;
            persist_anchors(P, u, tile);
            block_signal(P.doneA + u);
        } else if (phase == kItemP1) {
            if (!block_wait(P.doneA + u, (unsigned)P.nA, abort_flag, P.status, &s_flag, P.spin_limit)) break;
            if (u >= P.S && !block_wait(P.done2 + (u - P.S), n2, abort_flag, P.status, &s_flag, P.spin_limit))
                break;
            persist_p1<N2, N1>(smem, sp1, kp1, u, tile, P.S, P.SA);
            block_signal(P.done1 + u);
        } else {
            const unsigned need = n1 + (u == P.stall_unit ? 1u : 0u);
            if (!block_wait(P.done1 + u, need, abort_flag, P.status, &s_flag, P.spin_limit)) break;
            persist_p2<N2, N1>(smem, sp2, kp2, u, tile, P.S);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                s_old = atomicAdd(P.done2 + u, 1u);
            }
            __syncthreads();
            if (s_old == (unsigned)(n2 - 1) && threadIdx.x < 32) persist_peak<N2, N1>(P, u);
        }
    }
    (void)C2;
}

template <int N2, int N1>
size_t persist_smem() {
    constexpr int C1 = seqs_per_cta<N2>(N1);
    constexpr int C2 = seqs_per_cta<N1>(N2);
    const size_t a = pass_smem_bytes<N2, C1>(), b = pass_smem_bytes<N1, C2>();
    return a > b ? a : b;
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
