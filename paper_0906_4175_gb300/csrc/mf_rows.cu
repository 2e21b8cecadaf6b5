// mf_rows.cu -- pass 2 of the filter (row IFFTs + rho epilogue) as a
// persistent kernel in which a group of G warps owns whole rows: one warp for
// row length N1 = 1024 (N = 2^19, 2^20), two for N1 = 2048 (N = 2^21, 2^22).
//
// Row j2 of batch entry b is E[b N + j2 N1 .. + N1), contiguous.  Each group
// works through rows g, g + W, g + 2W, ... (W = groups in the grid) in its
// own shared-memory region:
//   1. wait for the row's bulk copy (cp.async.bulk, completion counted on the
//      group's mbarrier; bounded wait, status bit 1 and stop on expiry);
//   2. stage 0 (radix 32) from the staged row, written back in the padded
//      Stockham layout over the same region (then the middle stage, N1 = 2048);
//   3. the last stage reads the region, then -- before its arithmetic -- the
//      group's first thread starts the bulk copy of the group's next row into
//      the region, so the copy runs under the last stage and the epilogue;
//   4. epilogue as in the per-tile pass 2 (argmax with the lowest-j rule,
//      warp-aggregated trigger append), each warp's argmax of the row to
//      partials[unit][j2][warp of the group].
// The twiddle table is filled once per CTA; the stages of a row synchronise
// only its group (__syncwarp, or a named barrier for a pair of warps).
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

constexpr int kWarps = 8;                     // warps per CTA

// barrier of the G warps that own one row
template <int G>
struct GroupSync {
    static __device__ __forceinline__ void sync() {
        if constexpr (G == 1) {
            __syncwarp();
        } else {
            const unsigned id = 1u + (threadIdx.x >> 5) / G;   // named barriers 1.. (0 is __syncthreads)
            asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(32 * G) : "memory");
        }
    }
};

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
template <int L, int G>
struct GroupRhoSink {
    const RowsParams &p;
    const UnitInfo &u;
    const int j2;
    float bp = -1.f;
    int bj = 0x7fffffff;
    float2 bz = make_float2(0.f, 0.f);
    float2 *region;
    uint64_t *bar;
    const float2 *next_src;     // next row of this group, or NULL
    __device__ GroupRhoSink(const RowsParams &pp, const UnitInfo &uu, int jj, float2 *rg, uint64_t *br,
                            const float2 *nx)
        : p(pp), u(uu), j2(jj), region(rg), bar(br), next_src(nx) {}
    // the last stage has read the group's region: refill it with the next row
    __device__ __forceinline__ void after_loads() {
        GroupSync<G>::sync();
        fence_proxy_async();
        if (next_src != nullptr && (threadIdx.x & (32 * G - 1)) == 0) {
            mbar_expect_tx(bar, L * sizeof(float2));
            bulk_row_copy(region, next_src, L * sizeof(float2), bar);
        }
    }
    template <int R>
    __device__ __forceinline__ void store(int, int b, int stride, const float2 *v) {
        float pw[R];
#pragma unroll
        for (int r = 0; r < R; ++r) pw[r] = fmaf(v[r].x, v[r].x, v[r].y * v[r].y);
        const float m = tree_max0<R>(pw);
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

template <int L>
__device__ __forceinline__ const float2 *row_src(const RowsParams &p, int64_t r) {
    const int64_t n2 = (int64_t)1 << p.log2N2;
    const int64_t slot = r >> p.log2N2, j2 = r & (n2 - 1);
    return p.exch + (slot << p.log2N) + j2 * L;
}

}  // namespace

template <int L>
__global__ void __launch_bounds__(kWarps * 32, 2) k_pass2_rows(RowsParams p) {
    using S = FftShape<L>;
    constexpr int G = L / 1024;               // warps per row
    constexpr int NG = kWarps / G;            // rows in flight per CTA
    constexpr int T = L / 32;                 // threads per row (= 32 G)
    static_assert(G >= 1 && kWarps % G == 0 && T == 32 * G, "1024- or 2048-point rows");
    extern __shared__ __align__(16) float2 rows_smem[];
    __shared__ int gfail[NG];                 // a warp of the group gave up waiting
    float2 *tw = rows_smem + NG * S::STRIDE;
    uint64_t *bars = reinterpret_cast<uint64_t *>(tw + TwTable<L>::SIZE);
    const int grp = (threadIdx.x >> 5) / G, t = threadIdx.x & (T - 1), lane = threadIdx.x & 31;
    const int wig = (threadIdx.x >> 5) % G;   // warp within the group
    float2 *region = rows_smem + grp * S::STRIDE;
    fill_twiddles<L>(tw);
    if (t == 0) {
        mbar_init(&bars[grp], 1);
        gfail[grp] = 0;
    }
    mbar_fence_init();
    __syncthreads();
    const int64_t total = (int64_t)p.n_units << p.log2N2;
    const int64_t step = (int64_t)gridDim.x * NG;
    int64_t r = (int64_t)blockIdx.x * NG + grp;
    if (r < total && t == 0) {
        mbar_expect_tx(&bars[grp], L * sizeof(float2));
        bulk_row_copy(region, row_src<L>(p, r), L * sizeof(float2), &bars[grp]);
    }
    uint32_t parity = 0;
    for (; r < total; r += step) {
        // 1. the row has landed (bounded wait; every warp of the group waits on the same barrier)
        long long it = 0;
        bool ok = true;
        while (!mbar_try_wait(&bars[grp], parity)) {
            if (++it > p.spin_limit) { ok = false; break; }
        }
        ok = __all_sync(0xffffffffu, ok);
        if constexpr (G > 1) {   // the group leaves together: no warp may wait at a group barrier alone
            if (!ok && lane == 0) atomicOr(&gfail[grp], 1);
            GroupSync<G>::sync();
            ok = *(volatile int *)&gfail[grp] == 0;
        }
        if (!ok) {
            if (lane == 0) atomicOr(p.status, 2);
            return;   // the copy into this group's region never completed; nothing else is in flight
        }
        parity ^= 1u;
        const int slot = (int)(r >> p.log2N2);
        const int j2 = (int)(r & (((int64_t)1 << p.log2N2) - 1));
        const int unit = p.unit0 + slot;
        const UnitInfo u = p.units[unit];
        // 2. stage 0 from the staged row (element t + T q of the row at t + T q)
        float2 v[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) v[q] = region[t + T * q];
        Dft<32, +1>::run(v);
        GroupSync<G>::sync();
#pragma unroll
        for (int q = 0; q < 32; ++q) region[spad(32 * t + q)] = v[q];
        GroupSync<G>::sync();
        // 3./4. the remaining stages, next-row copy, epilogue
        const int64_t rn = r + step;
        GroupRhoSink<L, G> snk(p, u, j2, region, &bars[grp], rn < total ? row_src<L>(p, rn) : nullptr);
        if constexpr (S::NST == 2) {
            stockham_stage<L, S::R1, 32, +1, true, GroupRhoSink<L, G>, GroupSync<G>>(region, tw, 0, t, snk);
        } else {
            stockham_stage<L, S::R1, 32, +1, false, GroupRhoSink<L, G>, GroupSync<G>>(region, tw, 0, t, snk);
            stockham_stage<L, S::R2, 32 * S::R1, +1, true, GroupRhoSink<L, G>, GroupSync<G>>(
                region, tw + TwTable<L>::S1, 0, t, snk);
        }
        snk.finish(&p.partials[(((int64_t)unit << p.log2N2) + j2) * G + wig]);
    }
}

template <int L>
static size_t rows_smem() {
    return (size_t)(kWarps / (L / 1024)) * FftShape<L>::STRIDE * sizeof(float2) +
           (size_t)TwTable<L>::SIZE * sizeof(float2) + kWarps * sizeof(uint64_t);
}

bool pass2_rows_applies(int log2N) {
    const int lg1 = log2N - log2_n2(log2N);
    return lg1 == 10 || lg1 == 11;
}

int pass2_rows_partials(int log2N) {   // partials per unit: one per row and warp
    const int lg1 = log2N - log2_n2(log2N);
    return (1 << log2_n2(log2N)) * (lg1 == 11 ? 2 : 1);
}

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
    if (seg.log2N1 == 10) {
        int64_t grid = std::min<int64_t>(2 * (int64_t)n_sm, (rows + kWarps - 1) / kWarps);
        k_pass2_rows<1024><<<(unsigned)std::max<int64_t>(grid, 1), kWarps * 32, rows_smem<1024>(), st>>>(p);
    } else {
        int64_t grid = std::min<int64_t>(2 * (int64_t)n_sm, (rows + kWarps / 2 - 1) / (kWarps / 2));
        k_pass2_rows<2048><<<(unsigned)std::max<int64_t>(grid, 1), kWarps * 32, rows_smem<2048>(), st>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t rows_kernel_attributes() {
    {
        cudaError_t e0 = init_twiddle_tables();
        if (e0 != cudaSuccess) return e0;
    }
    cudaError_t e = cudaFuncSetAttribute(k_pass2_rows<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)rows_smem<1024>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_pass2_rows<2048>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)rows_smem<2048>());
}

}  // namespace mf
