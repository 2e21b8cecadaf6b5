// mf_pass1.cuh -- pieces of the staged pass 1 (template generation, weighting
// and column IFFTs with the next tile's inputs copied in under the current
// one) shared by the per-batch persistent pass-1 kernel (mf_pass1.cu) and the
// fused persistent scheduler (mf_fused.cu).
#pragma once
#include "mf_async.cuh"
#include "mf_filter.cuh"

namespace mf {

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

constexpr int kBoxRows = 64;   // rows of one W box (C x 64 complex64 = 4 KB at C = 8)

struct Pass1PfParams {
    const float2 *W;
    const UnitInfo *units;
    const float4 *anchors;
    const float *anchors4;
    float2 *E;
    int anc_stride, log2D, log2N;
    int unit0, n_items;
    int *status;                // bit 1: a bounded wait expired
    long long spin_limit;
};

template <int L, int C>
__host__ __device__ constexpr size_t pf_wbuf_elems() { return (size_t)(L / 2) * C; }

// twiddle entries kept in shared memory (see the layout above)
template <int L>
__host__ __device__ constexpr int pf_tw_elems() { return L == 1024 ? 17 * 32 : TwTable<L>::S1; }

template <int L, int C>
__host__ __device__ constexpr size_t pf_smem_bytes() {
    return pass_data_bytes<L, C>() + pf_wbuf_elems<L, C>() * sizeof(float2) +
           (size_t)(L / 2) * (sizeof(float4) + sizeof(float)) + (size_t)pf_tw_elems<L>() * sizeof(float2) +
           sizeof(uint64_t);
}

// The band fields of a unit (k_lo, k_hi, g_lo, n_anc: the first 16 bytes of
// its 32-byte-aligned UnitInfo), loaded a full item ahead of their use.
__device__ __forceinline__ int4 pf_band(const Pass1PfParams &p, int slot) {
    return __ldg(reinterpret_cast<const int4 *>(p.units + p.unit0 + slot));
}

// Start the copies of one item's inputs: the W rows n < L/2 of the tile's C
// columns and the anchor record of each row (anchor column kc / D, rows n,
// contiguous in the slot).  With a tensor map, thread 0 issues the TMA boxes
// of W that meet the band and bulk copies of the anchor rows in the band, all
// counted on bar (one phase per item); otherwise every thread copies 16-byte
// W chunks (skipped when both columns of a chunk are outside the band) and
// the anchor records of its rows with cp.async and commits one group.
// Called by all threads after a barrier that ends every read of the staging
// area.
template <int L, int C, int LG1, bool TMA>
__device__ __forceinline__ void pf_issue(const Pass1PfParams &p, const CUtensorMap *wmap, int item, int4 band,
                                         float2 *wbuf, float4 *abuf, float *abuf4, uint64_t *bar) {
    constexpr int NT = C * (L / 32);
    constexpr int TILES = (1 << LG1) / C;
    const int slot = item / TILES, tile = item - slot * TILES;
    const int k_lo = band.x, k_hi = band.y, g_lo = band.z, n_anc = band.w;
    const int kc = tile * C;
    const int gcol = kc >> p.log2D;
    const float4 *acol = p.anchors + (int64_t)slot * p.anc_stride + ((int64_t)gcol << (cx_ilog2(L) - 1));
    const float *acol4 = p.anchors4 + (int64_t)slot * p.anc_stride + ((int64_t)gcol << (cx_ilog2(L) - 1));
    if constexpr (TMA) {
        if (threadIdx.x == 0) {
            // rows holding a bin of the band: kc + C - 1 + n N1 >= k_lo and kc + n N1 < k_hi
            const int lo_num = k_lo - kc - (C - 1), hi_num = k_hi - kc;
            const int n_lo = lo_num <= 0 ? 0 : (lo_num + (1 << LG1) - 1) >> LG1;
            const int n_hi = hi_num <= 0 ? 0 : min(L / 2, (hi_num + (1 << LG1) - 1) >> LG1);
            fence_proxy_async();
            const bool in_range = MF_DBG(kc + C <= (1 << LG1) && ((int64_t)(gcol + 1) << (cx_ilog2(L) - 1)) <= p.anc_stride,
                                         kDbgCopy);
            if (n_hi > n_lo && in_range) {
                const int b0 = n_lo / kBoxRows, b1 = (n_hi + kBoxRows - 1) / kBoxRows;
                const int a0 = n_lo & ~3, a1 = (n_hi + 3) & ~3;   // 16-byte runs of the FP32 q4 terms
                mbar_expect_tx(bar, (uint32_t)((b1 - b0) * kBoxRows * C * sizeof(float2) +
                                               (n_hi - n_lo) * sizeof(float4) + (a1 - a0) * sizeof(float)));
                for (int b = b0; b < b1; ++b) tma_load_2d(wbuf + b * kBoxRows * C, wmap, kc, b * kBoxRows, bar);
                bulk_copy_g2s(abuf + n_lo, acol + n_lo, (uint32_t)((n_hi - n_lo) * sizeof(float4)), bar);
                bulk_copy_g2s(abuf4 + a0, acol4 + a0, (uint32_t)((a1 - a0) * sizeof(float)), bar);
            } else {
                mbar_arrive(bar);
            }
        }
    } else {
        constexpr int CH = C / 2;   // 16-byte chunks per row
#pragma unroll
        for (int i = 0; i < (L / 2) * CH / NT; ++i) {
            const int c = threadIdx.x + i * NT;
            const int n = c / CH, j = c - n * CH;
            const int k = kc + 2 * j + (n << LG1);
            if (k + 1 >= k_lo && k < k_hi) cp_async16(wbuf + n * C + 2 * j, p.W + k);
        }
        const int gstep = 1 << (LG1 - p.log2D);
        const int gbase = gcol - g_lo;
        for (int n = threadIdx.x; n < L / 2; n += NT) {
            const int a = gbase + n * gstep;
            if (a >= 0 && a < n_anc && MF_DBG(((int64_t)gcol << (cx_ilog2(L) - 1)) + n < p.anc_stride, kDbgAnchor)) {
                cp_async16(abuf + n, acol + n);
                cp_async4(abuf4 + n, acol4 + n);
            }
        }
        cp_async_commit();
    }
}

// 32-point DFT X_q = sum_r v_r e^{2 pi i r q / 32} of a vector whose only
// non-zero entry is x at r = rs < 16, given w = e^{2 pi i rs / 32}:
// X_q = x w^q for q < 8 by a running product, then X_{q+8} = i^rs X_q and
// X_{q+16} = (-1)^rs X_q, both exact.
__device__ __forceinline__ void dft32_single(float2 *v, float2 x, int rs, float2 w) {
    v[0] = x;
#pragma unroll
    for (int q = 1; q < 8; ++q) v[q] = cmul(v[q - 1], w);
    const int k = rs & 3;   // i^rs = c + i s
    const float c = k == 0 ? 1.f : (k == 2 ? -1.f : 0.f), s = k == 1 ? 1.f : (k == 3 ? -1.f : 0.f);
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q + 8] = make_float2(c * v[q].x - s * v[q].y, c * v[q].y + s * v[q].x);
    const float sg = (rs & 1) ? -1.f : 1.f;
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q + 16] = make_float2(sg * v[q].x, sg * v[q].y);
}

// Stage 1 of one column tile: template generation and weighting for this
// thread's 16 rows n = t + 32 r of column k1 = tile C + seq (warps skip groups
// of four rows outside every lane's band), the half-zero radix-32 DFT, and the
// store into the sequence's shared-memory column sq.  Reads the staged W tile,
// anchors and q4 terms.  NARROW (bands of a few rows, the chi^2 sub-bands):
// where no lane of the warp holds more than one row of the band, the DFT is
// dft32_single with w from the stage-1 table tw (exp(2 pi i r k / L), row L/64).
template <int L, int C, int LG1, bool NARROW = false>
__device__ __forceinline__ void pf_stage1(int tile, int seq, int t, int k_lo, int k_hi, int log2D,
                                          const float2 *wbuf, const float4 *abuf, const float *abuf4, float2 *sq,
                                          const float2 *tw = nullptr) {
    constexpr int T = L / 32;
    const int D = 1 << log2D;
    float2 v[32];
    const int k1 = tile * C + seq;
    const int k0 = k1 + (t << LG1);
    // offset from the anchor centre, the same on every row (D divides N1)
    const float d = (float)((k1 & (D - 1)) - (D >> 1));
    // rows r of this thread in the band: [rlo, rhi) (k grows with r)
    constexpr int LGS = cx_ilog2(T) + LG1;   // log2 of the row step T N1 in bins
    const int rlo = k_lo <= k0 ? 0 : min(16, (k_lo - k0 + (1 << LGS) - 1) >> LGS);
    const int rhi = k_hi <= k0 ? 0 : min(16, (k_hi - k0 + (1 << LGS) - 1) >> LGS);
    const int wlo = (int)__reduce_min_sync(0xffffffffu, (unsigned)rlo);
    const int whi = (int)__reduce_max_sync(0xffffffffu, (unsigned)rhi);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        if (4 * g + 4 > wlo && 4 * g < whi) {   // some lane of the warp has a bin of rows 4g..4g+3
#pragma unroll
            for (int r = 4 * g; r < 4 * g + 4; ++r) {
                const int n = t + r * T;
                const float2 w = wbuf[n * C + seq];
                const float4 a = abuf[n];
                const float a4 = abuf4[n];
                float ph = fmaf(fmaf(fmaf(fmaf(a4, d, a.w), d, a.z), d, a.y), d, a.x);
                ph -= rintf(ph);
                float sn, cs;
                __sincosf(6.283185307179586f * ph, &sn, &cs);
                const float2 x = make_float2(fmaf(w.x, cs, w.y * sn), fmaf(w.y, cs, -w.x * sn));  // W e^{-i 2 pi ph}
                v[r] = (r >= rlo && r < rhi) ? x : czero();   // staging outside the band is stale
            }
        } else {
#pragma unroll
            for (int r = 4 * g; r < 4 * g + 4; ++r) v[r] = czero();
        }
    }
    bool single = false;
    if constexpr (NARROW) {
        static_assert(L >= 512, "the row L/64 of the stage-1 table holds the 32nd roots for L >= 512");
        single = __reduce_max_sync(0xffffffffu, (unsigned)(rhi > rlo ? rhi - rlo : 0)) <= 1u;
        if (single) {
            float2 x = v[0];
#pragma unroll
            for (int r = 1; r < 16; ++r) x = cadd(x, v[r]);   // the one non-zero entry (or 0)
            const int rs = min(rlo, 15);
            dft32_single(v, x, rs, tw[(L / 64) * 32 + 2 * rs]);
        }
    }
    if (!single) dft32_halfzero<+1>(v);
#pragma unroll
    for (int r = 0; r < 32; ++r) sq[spad(32 * t + r)] = v[r];
}

}  // namespace mf
