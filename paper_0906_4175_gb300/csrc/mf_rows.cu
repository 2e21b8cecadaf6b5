// mf_rows.cu -- pass 2 of the filter (row IFFTs + rho epilogue) as a
// persistent kernel in which every warp owns whole rows, for row length
// N1 = 1024 (N = 2^19, 2^20).
//
// Row j2 of batch entry b is E[b N + j2 N1 .. + N1), 8 KiB contiguous.  Each
// warp works through rows w, w + W, w + 2W, ... (W = warps in the grid) in
// its own shared-memory region:
//   1. wait for the row's bulk copy (cp.async.bulk, completion counted on the
//      warp's mbarrier; bounded wait, status bit 1 and stop on expiry);
//   2. stage 0 (radix 32) from the staged row, written back in the padded
//      Stockham layout over the same region;
//   3. stage 1 reads the region, then -- before its arithmetic -- lane 0
//      starts the bulk copy of the warp's next row into the region, so the
//      copy runs under the last stage and the rho epilogue;
//   4. epilogue as in the per-tile pass 2 (argmax with the lowest-j rule,
//      warp-aggregated trigger append), the row's argmax to partials[unit][j2].
// The twiddle table is filled once per CTA; after start-up no CTA barrier is
// needed, since a row never leaves its warp.
#include "mf_filter.cuh"

namespace mf {

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_row_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
// orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy ones (the bulk copy refilling the region)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

constexpr int kL = 1024;                      // row length N1
constexpr int kWarps = 8;                     // warps (rows in flight) per CTA
using RowShape = FftShape<kL>;

struct RowsParams {
    const float2 *exch;
    const UnitInfo *units;
    float4 *partials;           // [unit][j2], N2 per unit
    mf_trigger *staged;
    uint64_t *keys;
    unsigned long long *counter;
    int64_t cap;
    int unit0, n_units;
    int log2N, log2N2, seg_idx;
    KeyLayout kl;
    int *status;
    long long spin_limit;
};

// epilogue of one row: per-butterfly argmax (lowest j on ties), triggers
struct WarpRhoSink {
    const RowsParams &p;
    const UnitInfo &u;
    const int j2;
    float bp = -1.f;
    int bj = 0x7fffffff;
    float2 bz = make_float2(0.f, 0.f);
    float2 *region;
    uint64_t *bar;
    const float2 *next_src;     // next row of this warp, or NULL
    __device__ WarpRhoSink(const RowsParams &pp, const UnitInfo &uu, int jj, float2 *rg, uint64_t *br,
                           const float2 *nx)
        : p(pp), u(uu), j2(jj), region(rg), bar(br), next_src(nx) {}
    // the last stage has read this warp's region: refill it with the next row
    __device__ __forceinline__ void after_loads() {
        __syncwarp();
        fence_proxy_async();
        if (next_src != nullptr && (threadIdx.x & 31) == 0) {
            mbar_expect_tx(bar, kL * sizeof(float2));
            bulk_row_copy(region, next_src, kL * sizeof(float2), bar);
        }
    }
    template <int R>
    __device__ __forceinline__ void store(int, int b, int stride, const float2 *v) {
        float pw[R];
        float m = 0.f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            pw[r] = fmaf(v[r].x, v[r].x, v[r].y * v[r].y);
            m = fmaxf(m, pw[r]);
        }
        if (m >= bp) {
            int rs = R - 1;
#pragma unroll
            for (int r = R - 2; r >= 0; --r) rs = (pw[r] == m) ? r : rs;
            const int j = j2 + ((b + rs * stride) << p.log2N2);
            if (m > bp || j < bj) {
                float2 z = v[R - 1];
#pragma unroll
                for (int r = R - 2; r >= 0; --r) z = (r == rs) ? v[r] : z;
                bp = m;
                bj = j;
                bz = z;
            }
        }
        if (__any_sync(0xffffffffu, m > u.thr2)) {
            const int lane = threadIdx.x & 31;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const bool pred = pw[r] > u.thr2;
                const unsigned msk = __ballot_sync(0xffffffffu, pred);
                if (msk == 0u) continue;
                const int leader = __ffs(msk) - 1;
                unsigned long long base = 0ull;
                if (lane == leader) base = atomicAdd(p.counter, (unsigned long long)__popc(msk));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (pred) {
                    const unsigned long long slot = base + (unsigned long long)__popc(msk & ((1u << lane) - 1u));
                    if (slot < (unsigned long long)p.cap) {
                        const int j = j2 + ((b + r * stride) << p.log2N2);
                        mf_trigger tr;
                        tr.tmpl = u.tmpl;
                        tr.seg = p.seg_idx;
                        tr.j = j;
                        tr.rho = sqrtf(pw[r]) * u.rho_scale;
                        tr.z_re = v[r].x * u.z_scale;
                        tr.z_im = v[r].y * u.z_scale;
                        p.staged[slot] = tr;
                        p.keys[slot] = ((uint64_t)u.tmpl << (p.kl.seg_bits + p.kl.j_bits)) |
                                       ((uint64_t)p.seg_idx << p.kl.j_bits) | (uint64_t)j;
                    }
                }
            }
        }
    }
    __device__ __forceinline__ void finish(float4 *out) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float op = __shfl_xor_sync(0xffffffffu, bp, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            const float ox = __shfl_xor_sync(0xffffffffu, bz.x, o);
            const float oy = __shfl_xor_sync(0xffffffffu, bz.y, o);
            if (op > bp || (op == bp && oj < bj)) { bp = op; bj = oj; bz = make_float2(ox, oy); }
        }
        if ((threadIdx.x & 31) == 0) *out = make_float4(bp, __int_as_float(bj), bz.x, bz.y);
    }
};

__device__ __forceinline__ const float2 *row_src(const RowsParams &p, int64_t r) {
    const int64_t n2 = (int64_t)1 << p.log2N2;
    const int64_t slot = r >> p.log2N2, j2 = r & (n2 - 1);
    return p.exch + (slot << p.log2N) + j2 * kL;
}

}  // namespace

__global__ void __launch_bounds__(kWarps * 32, 2) k_pass2_rows(RowsParams p) {
    extern __shared__ __align__(16) float2 rows_smem[];
    float2 *tw = rows_smem + kWarps * RowShape::STRIDE;
    uint64_t *bars = reinterpret_cast<uint64_t *>(tw + TwTable<kL>::SIZE);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 *region = rows_smem + warp * RowShape::STRIDE;
    fill_twiddles<kL>(tw);
    if (lane == 0) mbar_init(&bars[warp], 1);
    mbar_fence_init();
    __syncthreads();
    const int64_t total = (int64_t)p.n_units << p.log2N2;
    const int64_t step = (int64_t)gridDim.x * kWarps;
    int64_t r = (int64_t)blockIdx.x * kWarps + warp;
    if (r < total && lane == 0) {
        mbar_expect_tx(&bars[warp], kL * sizeof(float2));
        bulk_row_copy(region, row_src(p, r), kL * sizeof(float2), &bars[warp]);
    }
    uint32_t parity = 0;
    for (; r < total; r += step) {
        // 1. the row has landed (bounded wait)
        long long it = 0;
        bool ok = true;
        while (!mbar_try_wait(&bars[warp], parity)) {
            if (++it > p.spin_limit) { ok = false; break; }
        }
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) atomicOr(p.status, 2);
            return;   // the copy into this warp's region never completed; nothing else is in flight
        }
        parity ^= 1u;
        const int slot = (int)(r >> p.log2N2);
        const int j2 = (int)(r & (((int64_t)1 << p.log2N2) - 1));
        const int unit = p.unit0 + slot;
        const UnitInfo u = p.units[unit];
        // 2. stage 0 from the staged row (element t + 32 q of the row at t + 32 q)
        float2 v[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) v[q] = region[lane + 32 * q];
        Dft<32, +1>::run(v);
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 32; ++q) region[spad(32 * lane + q)] = v[q];
        __syncwarp();
        // 3./4. last stage, next-row copy, epilogue
        const int64_t rn = r + step;
        WarpRhoSink snk(p, u, j2, region, &bars[warp], rn < total ? row_src(p, rn) : nullptr);
        stockham_stage<kL, RowShape::R1, 32, +1, true>(region, tw, 0, lane, snk);
        snk.finish(&p.partials[((int64_t)unit << p.log2N2) + j2]);
    }
}

size_t pass2_rows_smem() {
    return (size_t)kWarps * RowShape::STRIDE * sizeof(float2) + (size_t)TwTable<kL>::SIZE * sizeof(float2) +
           kWarps * sizeof(uint64_t);
}

bool pass2_rows_applies(int log2N) { return log2N - log2_n2(log2N) == 10; }

cudaError_t launch_pass2_rows(const SegDev &seg, const UnitInfo *units, int unit0, int n_units, const float2 *exch,
                              float4 *partials, int seg_idx, KeyLayout kl, mf_trigger *staged, uint64_t *keys,
                              unsigned long long *counter, int64_t cap, int *status, long long spin_limit, int n_sm,
                              cudaStream_t st) {
    if (!pass2_rows_applies(seg.log2N)) return cudaErrorInvalidValue;
    RowsParams p;
    p.exch = exch;
    p.units = units;
    p.partials = partials;
    p.staged = staged;
    p.keys = keys;
    p.counter = counter;
    p.cap = cap;
    p.unit0 = unit0;
    p.n_units = n_units;
    p.log2N = seg.log2N;
    p.log2N2 = seg.log2N2;
    p.seg_idx = seg_idx;
    p.kl = kl;
    p.status = status;
    p.spin_limit = spin_limit;
    const int64_t rows = (int64_t)n_units << seg.log2N2;
    int64_t grid = std::min<int64_t>(2 * (int64_t)n_sm, (rows + kWarps - 1) / kWarps);
    if (grid < 1) grid = 1;
    k_pass2_rows<<<(unsigned)grid, kWarps * 32, pass2_rows_smem(), st>>>(p);
    return cudaGetLastError();
}

cudaError_t rows_kernel_attributes() {
    {
        cudaError_t e0 = init_twiddle_tables();
        if (e0 != cudaSuccess) return e0;
    }
    return cudaFuncSetAttribute(k_pass2_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pass2_rows_smem());
}

}  // namespace mf
