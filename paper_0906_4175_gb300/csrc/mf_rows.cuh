// mf_rows.cuh -- pieces of the warp-owned row pass (pass 2: row IFFTs + rho
// epilogue, one row per warp or warp pair, each row bulk-copied into the
// group's shared-memory region) shared by the per-batch rows kernel
// (mf_rows.cu) and the fused persistent scheduler (mf_fused.cu).
#pragma once
#include "mf_async.cuh"
#include "mf_filter.cuh"

namespace mf {

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
    int stall_unit;             // test hook: rows of this unit never arrive (bounded-wait tests), -1 = none
};

// epilogue of one row: per-butterfly argmax (lowest j on ties), triggers.
// FULL = false keeps only the row's largest |raw|^2 (the sample and z of the
// peak are found afterwards by k_peaks_rows, which recomputes the winning
// rows): the per-thread index and z search is the costliest part of the
// epilogue, and it would run on every row for one peak per template.
template <int L, int G, bool FULL = true>
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
            bulk_copy_g2s(region, next_src, L * sizeof(float2), bar);
        }
    }
    template <int R>
    __device__ __forceinline__ void store(int, int b, int stride, const float2 *v) {
        float pw[R];
#pragma unroll
        for (int r = 0; r < R; ++r) pw[r] = fmaf(v[r].x, v[r].x, v[r].y * v[r].y);
        const float m = tree_max0<R>(pw);
        if constexpr (!FULL) {
            bp = fmaxf(bp, m);
        } else if (m >= bp) {
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
        if constexpr (!FULL) {   // the row's largest |raw|^2 only (j = -1: found later)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bp = fmaxf(bp, __shfl_xor_sync(0xffffffffu, bp, o));
            if ((threadIdx.x & 31) == 0) *out = make_float4(bp, __int_as_float(-1), 0.f, 0.f);
            return;
        }
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

// the test hook's unit: the FP32 rows kernel withholds its row copies, the
// tensor-core kernel its MMA commits
__device__ __forceinline__ bool row_withheld(const RowsParams &p, int64_t r) {
    return p.unit0 + (int)(r >> p.log2N2) == p.stall_unit;
}

template <int L>
__device__ __forceinline__ const float2 *row_src(const RowsParams &p, int64_t r) {
    const int64_t n2 = (int64_t)1 << p.log2N2;
    const int64_t slot = r >> p.log2N2, j2 = r & (n2 - 1);
    if (!MF_DBG(slot < p.n_units && r >= 0 && (j2 + 1) * L <= ((int64_t)1 << p.log2N), kDbgRows))
        return p.exch;   // a valid row, so the copy stays inside the exchange
    return p.exch + (slot << p.log2N) + j2 * L;
}

template <int L>
inline size_t rows_smem() {
    return (size_t)(kWarps / (L / 1024)) * FftShape<L>::STRIDE * sizeof(float2) +
           (size_t)TwTable<L>::SIZE * sizeof(float2) + kWarps * sizeof(uint64_t);
}


}  // namespace mf
