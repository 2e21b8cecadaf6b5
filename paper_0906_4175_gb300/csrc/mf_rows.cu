// mf_rows.cu -- pass 2 of the filter (row IFFTs + rho epilogue) as
// persistent kernels in which a group of warps owns whole rows: one warp for
// row length N1 = 1024 (N = 2^19, 2^20), two for N1 = 2048 (N = 2^21, 2^22,
// and the 512 x 2048 split of 2^20), four for N1 = 4096 (the 1024 x 4096
// split of 2^22).
//
// Row j2 of batch entry b is E[b N + j2 N1 .. + N1), contiguous.  Each group
// works through rows g, g + W, g + 2W, ... (W = groups in the grid) in its
// own shared-memory region:
//   1. wait for the row's bulk copy (cp.async.bulk, completion counted on the
//      group's mbarrier; bounded wait, status bit 1 and stop on expiry);
//   2. stage 0 (radix 32) from the staged row, written back in the padded
//      Stockham layout over the same region;
//   3. the remaining stages (k_pass2_rows, k_pass2_rows_group below); once the
//      region has been read for the last time, the group's first thread
//      starts the bulk copy of the group's next row into it, so the copy runs
//      under the remaining arithmetic and the epilogue;
//   4. epilogue as in the per-tile pass 2 (argmax with the lowest-j rule,
//      warp-aggregated trigger append), each warp's argmax of the row to
//      partials[unit][j2][warp of the group].
// The twiddle tables are copied once per CTA; the stages of a row synchronise
// only its group (__syncwarp, or a named barrier for a pair of warps).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mf_rows.cuh"

namespace mf {

// 1024-point rows, one warp per row: stage 0, then the last stage with the
// next row's copy started from the sink once the region has been read.
// FULL = false: each row's partial holds only its largest |raw|^2 (k_peaks_rows
// then finds the peak's sample and z).
template <int L, bool FULL>
__global__ void __launch_bounds__(kWarps * 32, 2) k_pass2_rows(RowsParams p) {
    using S = FftShape<L>;
    static_assert(L == 1024 && S::NST == 2 && S::T == 32, "1024-point rows (one warp each)");
    constexpr int G = 1, T = 32;
    extern __shared__ __align__(16) float2 rows_smem[];
    float2 *tw = rows_smem + kWarps * S::STRIDE;
    uint64_t *bars = reinterpret_cast<uint64_t *>(tw + TwTable<L>::SIZE);
    const int grp = threadIdx.x >> 5, t = threadIdx.x & (T - 1);
    float2 *region = rows_smem + grp * S::STRIDE;
    fill_twiddles<L>(tw);
    if (t == 0) mbar_init(&bars[grp], 1);
    mbar_fence_init();
    __syncthreads();
    const int64_t total = (int64_t)p.n_units << p.log2N2;
    const int64_t step = (int64_t)gridDim.x * kWarps;
    int64_t r = (int64_t)blockIdx.x * kWarps + grp;
    if (r < total && t == 0 && !row_withheld(p, r)) {
        mbar_expect_tx(&bars[grp], L * sizeof(float2));
        bulk_copy_g2s(region, row_src<L>(p, r), L * sizeof(float2), &bars[grp]);
    }
    uint32_t parity = 0;
    for (; r < total; r += step) {
        // 1. the row has landed (bounded wait)
        long long it = 0;
        bool ok = true;
        while (!mbar_try_wait(&bars[grp], parity)) {
            if (++it > p.spin_limit) { ok = false; break; }
        }
        if (!__all_sync(0xffffffffu, ok)) {
            if (t == 0) atomicOr(p.status, 2);
            return;   // the copy into this warp's region never completed; nothing else is in flight
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
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 32; ++q) region[spad(32 * t + q)] = v[q];
        __syncwarp();
        // 3./4. the last stage, next-row copy, epilogue
        const int64_t rn = r + step;
        GroupRhoSink<L, G, FULL> snk(p, u, j2, region, &bars[grp],
                                     rn < total && !row_withheld(p, rn) ? row_src<L>(p, rn) : nullptr);
        stockham_stage<L, S::R1, 32, +1, true, GroupRhoSink<L, G, FULL>, GroupSync<G>>(region, tw, 0, t, snk);
        if (MF_DBG(slot < p.n_units && j2 < (1 << p.log2N2), kDbgRows))
            snk.finish(&p.partials[((int64_t)unit << p.log2N2) + j2]);
    }
}

// ---------------------------------------------------------------------------
// Peaks of a batch after k_pass2_rows<1024, false>: one warp per unit.  M = the
// largest of the unit's row maxima; every row whose maximum equals M (one,
// unless rows tie) is transformed again from the exchange, with the very
// arithmetic of k_pass2_rows (stage 0, the padded write, the last stage with
// the same table), and the lowest sample j with |raw|^2 == M gives the peak's
// j and z -- the record the per-row argmax would have produced.
// ---------------------------------------------------------------------------
struct CaptureSink {
    float2 v[32];
    template <int R>
    __device__ __forceinline__ void store(int, int, int, const float2 *x) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x[r];
    }
};

__global__ void __launch_bounds__(kWarps * 32) k_peaks_rows(const float2 *__restrict__ exch,
                                                            const UnitInfo *__restrict__ units, int unit0,
                                                            int n_units, int n_all, int log2N, int log2N2,
                                                            const float4 *__restrict__ partials, int seg_idx,
                                                            int n_seg, mf_peak *__restrict__ peaks) {
    constexpr int L = 1024;
    using S = FftShape<L>;
    extern __shared__ __align__(16) float2 rows_smem[];
    float2 *tw = rows_smem + kWarps * S::STRIDE;
    const int w = threadIdx.x >> 5, t = threadIdx.x & 31;
    float2 *region = rows_smem + w * S::STRIDE;
    fill_twiddles<L>(tw);
    __syncthreads();
    const int b = blockIdx.x * kWarps + w;   // unit within the batch
    if (b >= n_units) return;
    const int unit = unit0 + b;
    const int n2 = 1 << log2N2;
    const float4 *pp = partials + ((int64_t)unit << log2N2);
    float M = -1.f;
    for (int j2 = t; j2 < n2; j2 += 32) M = fmaxf(M, pp[j2].x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) M = fmaxf(M, __shfl_xor_sync(0xffffffffu, M, o));
    int bj = 0x7fffffff;
    float2 bz = make_float2(0.f, 0.f);
    for (int r0 = 0; r0 < n2; r0 += 32) {
        unsigned cand = __ballot_sync(0xffffffffu, pp[r0 + t].x == M);
        while (cand != 0u) {
            const int j2 = r0 + __ffs(cand) - 1;
            cand &= cand - 1u;
            if (!MF_DBG(b < n_units && (int64_t)(j2 + 1) * L <= ((int64_t)1 << log2N), kDbgRows)) continue;
            const float2 *row = exch + ((int64_t)b << log2N) + (int64_t)j2 * L;
            float2 v[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = row[t + 32 * q];
            Dft<32, +1>::run(v);
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 32; ++q) region[spad(32 * t + q)] = v[q];
            __syncwarp();
            CaptureSink cs;
            stockham_stage<L, S::R1, 32, +1, true, CaptureSink, GroupSync<1>>(region, tw, 0, t, cs);
#pragma unroll
            for (int r = 0; r < 32; ++r) {   // outputs t + 32 r of the row (j increases with r)
                const float pw = fmaf(cs.v[r].x, cs.v[r].x, cs.v[r].y * cs.v[r].y);
                const int j = j2 + ((t + 32 * r) << log2N2);
                if (pw == M && j < bj) {
                    bj = j;
                    bz = cs.v[r];
                }
            }
            __syncwarp();   // the region is read before the next candidate row overwrites it
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        const float ox = __shfl_xor_sync(0xffffffffu, bz.x, o);
        const float oy = __shfl_xor_sync(0xffffffffu, bz.y, o);
        if (oj < bj) {
            bj = oj;
            bz = make_float2(ox, oy);
        }
    }
    if (t == 0) {
        const UnitInfo u = units[unit];
        mf_peak pk;
        pk.rho = sqrtf(M) * u.rho_scale;
        pk.j = bj;
        pk.z_re = bz.x * u.z_scale;
        pk.z_im = bz.y * u.z_scale;
        if (MF_DBG(u.tmpl >= 0 && u.tmpl < n_all && seg_idx < n_seg, kDbgOut))
            peaks[(int64_t)u.tmpl * n_seg + seg_idx] = pk;
    }
}

// ---------------------------------------------------------------------------
// Rows of L = 1024 G points on a group of G = 2 or 4 warps: 2048-point rows
// (N = 2^21, 2^22, and the 512 x 2048 split of 2^20) and 4096-point rows (the
// 1024 x 4096 split of 2^22), with the arithmetic of the radix 32 x 32 x G
// Stockham schedule of the per-tile kernel (bit-identical) but one
// shared-memory round trip fewer.  Stages 0 and 1 run as in the generic
// schedule; after stage 1, lane k of warp h holds z[1024 h + k + 32 r]
// (r < 32), the 1024-point transform of the samples n = h (mod G).  The last
// stage, for b = k + 32 r < 1024 and q < G,
//   X[b + 1024 q] = sum_p w^(p b) z[1024 p + b] e^(2 pi i p q / G),
// w = exp(2 pi i / L), needs lane k of every warp: warp h takes the
// RW = 32 / G values of r in [RW h, RW h + RW) and receives the other warps'
// values there through the front of the group's region (stage 1 has read it
// by then); the next row's copy starts once that exchange has been read.
// Shared memory keeps the stage-1 table and rows p = 1 .. G - 1 of the last
// stage's table.  Pass 2 at N = 2^21: 4.2 us per template against 4.9 for
// the generic three-stage row form; a separate exchange area, with the copy
// started right after stage 1's loads, needs the twiddles read through L1 to
// keep two CTAs per SM and measured 4.7.
// ---------------------------------------------------------------------------
template <int G>
__host__ __device__ constexpr size_t rows_group_smem() {
    return (size_t)(kWarps / G) * FftShape<1024 * G>::STRIDE * sizeof(float2) + (size_t)1024 * G * sizeof(float2) +
           (kWarps / G) * sizeof(uint64_t);
}

// The transform of one landed row by its group (all G warps): stage 0 from
// the unpadded row in the region, stages 1 and the radix-G last stage through
// the region, outputs o[q][i] = X[b + 1024 q], b = k + 32 (RW h + i).  gfail:
// the group's wait flag, checked once every warp has read the row (the group
// then leaves: returns false); the region is free when it returns.
template <int G>
__device__ __forceinline__ bool group_row(float2 *region, const float2 *tw1, const float2 *tw2, int h, int lane,
                                          const volatile int *gfail, float2 (&o)[G][32 / G]) {
    constexpr int L = 1024 * G, T = 32 * G, RW = 32 / G;
    const int t = 32 * h + lane;
    float2 *xb = region;   // the exchange, once stage 1 has read the region
    // stage 0 (radix 32, Ns = 1): butterfly t reads x[t + T q]
    // (after a wait that ran out the region is stale; the group leaves together at the barrier below)
    float2 v[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = region[t + T * q];
    Dft<32, +1>::run(v);
    GroupSync<G>::sync();   // every read of the landed row is done; gfail is final
    if (gfail != nullptr && *gfail != 0) return false;
#pragma unroll
    for (int q = 0; q < 32; ++q) region[spad(32 * t + q)] = v[q];
    GroupSync<G>::sync();
    // stage 1 (radix 32, Ns = 32): butterfly t = 32 h + k reads y[t + T r]
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = region[spad(t + T * q)];
    GroupSync<G>::sync();   // the exchange below overwrites the region
#pragma unroll
    for (int q = 1; q < 32; ++q) v[q] = cmul(v[q], tw1[q * 32 + lane]);
    Dft<32, +1>::run(v);
    // exchange: slot ((src G + dst) RW + i) 32 + k holds z_src[k + 32 (RW dst + i)]
#pragma unroll
    for (int d = 0; d < G; ++d) {
        if (d == h) continue;
#pragma unroll
        for (int i = 0; i < RW; ++i) xb[((h * G + d) * RW + i) * 32 + lane] = v[RW * d + i];
    }
    GroupSync<G>::sync();
#pragma unroll
    for (int i = 0; i < RW; ++i) {
        const int b = lane + 32 * (RW * h + i);
        float2 x[G];
#pragma unroll
        for (int q = 0; q < G; ++q) x[q] = q == h ? v[RW * h + i] : xb[((q * G + h) * RW + i) * 32 + lane];
#pragma unroll
        for (int q = 1; q < G; ++q) x[q] = cmul(x[q], tw2[(q - 1) * 1024 + b]);
        Dft<G, +1>::run(x);
#pragma unroll
        for (int q = 0; q < G; ++q) o[q][i] = x[q];
    }
    GroupSync<G>::sync();   // every read of the region is done
    static_assert(L == 1024 * G, "row length");
    return true;
}

template <int G, bool FULL>
__global__ void __launch_bounds__(kWarps * 32, 2) k_pass2_rows_group(RowsParams p) {
    constexpr int L = 1024 * G, NG = kWarps / G, T = 32 * G, RW = 32 / G;
    using S = FftShape<L>;
    static_assert((G == 2 || G == 4) && S::NST == 3 && S::R2 == G && S::T == T, "rows of 2048 or 4096 points");
    static_assert(G * G * RW * 32 <= S::STRIDE, "the exchange fits the row region");
    extern __shared__ __align__(16) float2 rows_smem[];
    __shared__ int gfail[NG];
    const int grp = (threadIdx.x >> 5) / G, t = threadIdx.x & (T - 1), lane = threadIdx.x & 31;
    const int h = (threadIdx.x >> 5) % G;                     // warp within the group
    float2 *region = rows_smem + grp * S::STRIDE;
    float2 *tw1 = rows_smem + NG * S::STRIDE;                   // stage 1: [r 32 + k] = exp(2 pi i r k / 1024)
    float2 *tw2 = tw1 + 1024;                                   // last stage: [(p - 1) 1024 + b] = w^(p b)
    uint64_t *bars = reinterpret_cast<uint64_t *>(tw2 + 1024 * (G - 1));
    {
        const float2 *src = g_tw_tables + tw_offset<L>();
        for (int m = threadIdx.x; m < 1024 * G; m += blockDim.x)   // rows p >= 1 of the last stage's table
            tw1[m] = __ldg(&src[m < 1024 ? m : TwTable<L>::S1 + m]);
    }
    if (t == 0) {
        mbar_init(&bars[grp], 1);
        gfail[grp] = 0;
    }
    mbar_fence_init();
    __syncthreads();
    const int64_t total = (int64_t)p.n_units << p.log2N2;
    const int64_t step = (int64_t)gridDim.x * NG;
    int64_t r = (int64_t)blockIdx.x * NG + grp;
    if (r < total && t == 0 && !row_withheld(p, r)) {
        mbar_expect_tx(&bars[grp], L * sizeof(float2));
        bulk_copy_g2s(region, row_src<L>(p, r), L * sizeof(float2), &bars[grp]);
    }
    uint32_t parity = 0;
    for (; r < total; r += step) {
        long long it = 0;
        bool ok = true;
        while (!mbar_try_wait_sleep(&bars[grp], parity, 500u)) {
            if (++it > p.spin_limit) { ok = false; break; }
        }
        ok = __all_sync(0xffffffffu, ok);
        if (!ok && lane == 0) atomicOr(&gfail[grp], 1);
        parity ^= 1u;
        const int slot = (int)(r >> p.log2N2);
        const int j2 = (int)(r & (((int64_t)1 << p.log2N2) - 1));
        const int unit = p.unit0 + slot;
        const UnitInfo u = p.units[unit];
        const int64_t rn = r + step;
        const float2 *next = rn < total && !row_withheld(p, rn) ? row_src<L>(p, rn) : nullptr;
        float2 o[G][RW];
        if (!group_row<G>(region, tw1, tw2, h, lane, &gfail[grp], o)) {
            if (lane == 0) atomicOr(p.status, 2);
            return;   // the copy into this group's region never completed; nothing else is in flight
        }
        // every read of the region is done: start the next row's copy
        fence_proxy_async();
        if (next != nullptr && t == 0) {
            mbar_expect_tx(&bars[grp], L * sizeof(float2));
            bulk_copy_g2s(region, next, L * sizeof(float2), &bars[grp]);
        }
        // epilogue: outputs b + 1024 q, b = k + 32 (RW h + i)
        GroupRhoSink<L, G, FULL> snk(p, u, j2, region, &bars[grp], nullptr);
#pragma unroll
        for (int q = 0; q < G; ++q) snk.template store<RW>(0, lane + 32 * RW * h + 1024 * q, 32, o[q]);
        if (MF_DBG(slot < p.n_units && j2 < (1 << p.log2N2), kDbgRows))
            snk.finish(&p.partials[(((int64_t)unit << p.log2N2) + j2) * G + h]);
    }
}

// Peaks of a batch after k_pass2_rows_group<G, false>: one group of G warps
// per unit, as k_peaks_rows does for 1024-point rows -- M = the largest of the
// unit's row maxima (G partials per row), and every row that reaches it is
// loaded into the group's region and transformed again by group_row, the
// code of the row kernel, for the lowest sample with |raw|^2 == M.
template <int G>
__global__ void __launch_bounds__(kWarps * 32) k_peaks_rows_group(const float2 *__restrict__ exch,
                                                                  const UnitInfo *__restrict__ units, int unit0,
                                                                  int n_units, int n_all, int log2N, int log2N2,
                                                                  const float4 *__restrict__ partials, int seg_idx,
                                                                  int n_seg, mf_peak *__restrict__ peaks) {
    constexpr int L = 1024 * G, NG = kWarps / G, T = 32 * G, RW = 32 / G;
    using S = FftShape<L>;
    extern __shared__ __align__(16) float2 rows_smem[];
    __shared__ int s_j[kWarps];
    __shared__ float2 s_z[kWarps];
    const int grp = (threadIdx.x >> 5) / G, t = threadIdx.x & (T - 1), lane = threadIdx.x & 31;
    const int h = (threadIdx.x >> 5) % G;
    float2 *region = rows_smem + grp * S::STRIDE;
    float2 *tw1 = rows_smem + NG * S::STRIDE;
    float2 *tw2 = tw1 + 1024;
    {
        const float2 *src = g_tw_tables + tw_offset<L>();
        for (int m = threadIdx.x; m < 1024 * G; m += blockDim.x)
            tw1[m] = __ldg(&src[m < 1024 ? m : TwTable<L>::S1 + m]);
    }
    __syncthreads();
    const int b = blockIdx.x * NG + grp;   // unit within the batch (the group's warps agree)
    if (b >= n_units) return;              // whole groups leave: no group barrier is left waiting
    const int unit = unit0 + b;
    const int n2 = 1 << log2N2;
    const float4 *pp = partials + ((int64_t)unit << log2N2) * G;
    // every warp of the group computes M and the candidate rows itself (same values)
    float M = -1.f;
    for (int e = lane; e < n2 * G; e += 32) M = fmaxf(M, pp[e].x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) M = fmaxf(M, __shfl_xor_sync(0xffffffffu, M, o));
    int bj = 0x7fffffff;
    float2 bz = make_float2(0.f, 0.f);
    for (int r0 = 0; r0 < n2; r0 += 32) {
        float rm = -1.f;
#pragma unroll
        for (int q = 0; q < G; ++q) rm = fmaxf(rm, pp[(int64_t)(r0 + lane) * G + q].x);
        unsigned cand = __ballot_sync(0xffffffffu, rm == M);
        while (cand != 0u) {
            const int j2 = r0 + __ffs(cand) - 1;
            cand &= cand - 1u;
            const bool in_range = MF_DBG(b < n_units && (int64_t)(j2 + 1) * L <= ((int64_t)1 << log2N), kDbgRows);
            const float2 *row = exch + ((int64_t)b << log2N) + (in_range ? (int64_t)j2 * L : 0);
            for (int e = t; e < L; e += T) region[e] = row[e];   // the row as its bulk copy lands it
            GroupSync<G>::sync();
            float2 o[G][RW];
            group_row<G>(region, tw1, tw2, h, lane, nullptr, o);
#pragma unroll
            for (int q = 0; q < G; ++q)
#pragma unroll
                for (int i = 0; i < RW; ++i) {   // output b + 1024 q, b = k + 32 (RW h + i)
                    const float pw = fmaf(o[q][i].x, o[q][i].x, o[q][i].y * o[q][i].y);
                    const int j = j2 + ((lane + 32 * (RW * h + i) + 1024 * q) << log2N2);
                    if (in_range && pw == M && j < bj) {
                        bj = j;
                        bz = o[q][i];
                    }
                }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        const float ox = __shfl_xor_sync(0xffffffffu, bz.x, o);
        const float oy = __shfl_xor_sync(0xffffffffu, bz.y, o);
        if (oj < bj) {
            bj = oj;
            bz = make_float2(ox, oy);
        }
    }
    const int wi = threadIdx.x >> 5;
    if (lane == 0) {
        s_j[wi] = bj;
        s_z[wi] = bz;
    }
    GroupSync<G>::sync();
    if (h == 0 && lane == 0) {
        for (int q = 1; q < G; ++q)
            if (s_j[wi + q] < bj) {
                bj = s_j[wi + q];
                bz = s_z[wi + q];
            }
        const UnitInfo u = units[unit];
        mf_peak pk;
        pk.rho = sqrtf(M) * u.rho_scale;
        pk.j = bj;
        pk.z_re = bz.x * u.z_scale;
        pk.z_im = bz.y * u.z_scale;
        if (MF_DBG(u.tmpl >= 0 && u.tmpl < n_all && seg_idx < n_seg, kDbgOut))
            peaks[(int64_t)u.tmpl * n_seg + seg_idx] = pk;
    }
}

// ---------------------------------------------------------------------------
// Tensor-core form of the 1024-point rows (fft_mode MF_FFT_TC_FP16 /
// MF_FFT_TC_BF16).  Stage 0 of a row is Y_t[p] = sum_q x[t + 32 q] w^(pq),
// w = exp(2 pi i / 32), t, p, q < 32: for each row the complex product of the
// 32 x 32 matrix X[t][q] with the DFT matrix.  The four warps 4g .. 4g + 3 of
// a CTA form one tile of M = 128 GEMM rows (warp, t), K = 64 (re, im of the
// 32 inputs), N = 64 (re, im of the 32 outputs), with B the real form of the
// DFT matrix: B[2q][2p] = B[2q+1][2p+1] = cos, B[2q][2p+1] = -B[2q+1][2p] = sin.
// A and B are split into 16-bit hi + lo parts and D = A_hi B_hi + A_hi B_lo +
// A_lo B_hi is accumulated in FP32 in tensor memory (tcgen05.mma kind::f16,
// 3 x 4 instructions of K = 16 issued by one thread of the tile, completion
// on an mbarrier); each warp reads its 32 lanes back with tcgen05.ld and goes
// on with the FP32 second stage and the rho epilogue of the FP32 kernel.
// FP16 rows are scaled by a power of two (max |x| in [2^14, 2^15)) before the
// split and unscaled after; BF16 has the FP32 exponent range.
// Shared-memory operands use the no-swizzle K-major canonical layout: core
// matrices of 8 rows x 16 bytes, LBO = 128 B between K-adjacent ones, SBO
// between 8-row groups.  A warp's row region (8448 B) holds, per 8 rows of t,
// [A_hi 1 KB | A_lo 1 KB | 64 B], so the tile's SBO is 2112 B; B^T is 64 x 64
// (SBO 1 KB) for hi and lo.
// ---------------------------------------------------------------------------
constexpr int kTcRegion = 1056;               // float2 per warp region = 8448 B = 4 x 2112 B
constexpr uint32_t kTcSboA = 2112, kTcLbo = 128, kTcSboB = 1024, kTcBBytes = 2 * 64 * 64 * 2;
constexpr int kTcCols = 64;                   // TMEM columns per tile (N = 64 FP32)

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);   // version 1, no swizzle
}

// 16-bit split of a pair: hi = round(a), lo = round(a - hi) packed as 2 x 16 bits
template <int TCM>
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
    if constexpr (TCM == MF_FFT_TC_BF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    } else {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
}

template <int TCM>
__device__ __forceinline__ void store16(uint8_t *p, float v) {
    if constexpr (TCM == MF_FFT_TC_BF16) *reinterpret_cast<__nv_bfloat16 *>(p) = __float2bfloat16_rn(v);
    else *reinterpret_cast<__half *>(p) = __float2half_rn(v);
}
template <int TCM>
__device__ __forceinline__ float round16(float v) {
    if constexpr (TCM == MF_FFT_TC_BF16) return __bfloat162float(__float2bfloat16_rn(v));
    else return __half2float(__float2half_rn(v));
}

__device__ __forceinline__ void tile_sync(int g) {   // the 4 warps of tile g (named barrier 1 + g)
    asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory");
}

template <int TCM>
__global__ void __launch_bounds__(kWarps * 32, 2) k_pass2_rows_tc(RowsParams p) {
    constexpr int L = 1024;
    extern __shared__ __align__(16) float2 rows_smem[];
    __shared__ int gfail[2];
    __shared__ uint32_t tmem_base;
    float2 *tw = rows_smem + kWarps * kTcRegion;
    uint8_t *Bm = reinterpret_cast<uint8_t *>(tw + TwTable<L>::SIZE);
    uint64_t *bars = reinterpret_cast<uint64_t *>(Bm + kTcBBytes);   // kWarps row barriers, 2 tile barriers
    const int w = threadIdx.x >> 5, t = threadIdx.x & 31, g = w >> 2, rl = w & 3;
    float2 *region = rows_smem + w * kTcRegion;
    fill_twiddles<L>(tw);
    // B^T[n][k] of the DFT matrix, hi at Bm, lo at Bm + 8 KB
    for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
        const int n = e >> 6, k = e & 63, pp = n >> 1, q = k >> 1;
        double sn, cs;
        sincospi((double)((pp * q) & 31) / 16.0, &sn, &cs);
        const float v = (float)((n & 1) == 0 ? ((k & 1) == 0 ? cs : -sn) : ((k & 1) == 0 ? sn : cs));
        const uint32_t off = (n >> 3) * kTcSboB + (k >> 3) * kTcLbo + (n & 7) * 16 + (k & 7) * 2;
        store16<TCM>(Bm + off, v);
        store16<TCM>(Bm + 8192 + off, v - round16<TCM>(v));
    }
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(2 * kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) mbar_init(&bars[w], 1);
    if (threadIdx.x == 0) {
        mbar_init(&bars[kWarps], 1);
        mbar_init(&bars[kWarps + 1], 1);
        gfail[0] = gfail[1] = 0;
    }
    mbar_fence_init();
    fence_proxy_async();   // B, written by this CTA's threads, is read by the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base + (uint32_t)(kTcCols * g);
    const int64_t total = (int64_t)p.n_units << p.log2N2;
    const int64_t step = (int64_t)gridDim.x * kWarps;
    int64_t r0 = (int64_t)blockIdx.x * kWarps + 4 * g;   // the tile's first row; rows r0 .. r0 + 3 go together
    if (r0 + rl < total && t == 0) {
        mbar_expect_tx(&bars[w], L * sizeof(float2));
        bulk_copy_g2s(region, row_src<L>(p, r0 + rl), L * sizeof(float2), &bars[w]);
    }
    uint32_t parity = 0, tparity = 0;
    for (; r0 < total; r0 += step) {
        const int64_t r = r0 + rl;
        const bool has = r < total;
        // 1. the row has landed (bounded wait); the tile leaves together on expiry
        bool ok = true;
        if (has) {
            long long it = 0;
            while (!mbar_try_wait(&bars[w], parity)) {
                if (++it > p.spin_limit) { ok = false; break; }
            }
            ok = __all_sync(0xffffffffu, ok);
            parity ^= 1u;
        }
        if (!ok && t == 0) atomicOr(&gfail[g], 1);
        tile_sync(g);
        if (*(volatile int *)&gfail[g] != 0) {
            if (t == 0 && !ok) atomicOr(p.status, 2);
            break;
        }
        // 2. this warp's 32 GEMM rows: x[t + 32 q], split into hi + lo
        float2 v[32];
        float unscale = 1.f;
        if (has) {
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = region[t + 32 * q];
            if constexpr (TCM == MF_FFT_TC_FP16) {
                float m = 0.f;
#pragma unroll
                for (int q = 0; q < 32; ++q) m = fmaxf(m, fmaxf(fabsf(v[q].x), fabsf(v[q].y)));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                if (m > 0.f && m < 3.0e38f) {
                    const int e = 14 - ilogbf(m);
                    const float s = ldexpf(1.f, e);
                    unscale = ldexpf(1.f, -e);
#pragma unroll
                    for (int q = 0; q < 32; ++q) v[q] = make_float2(v[q].x * s, v[q].y * s);
                }
            }
            __syncwarp();   // every lane has read the staged row
            uint8_t *blk = reinterpret_cast<uint8_t *>(region) + (t >> 3) * kTcSboA + (t & 7) * 16;
#pragma unroll
            for (int j = 0; j < 8; ++j) {   // inputs q = 4j .. 4j + 3
                uint4 h, l;
                split2<TCM>(v[4 * j].x, v[4 * j].y, h.x, l.x);
                split2<TCM>(v[4 * j + 1].x, v[4 * j + 1].y, h.y, l.y);
                split2<TCM>(v[4 * j + 2].x, v[4 * j + 2].y, h.z, l.z);
                split2<TCM>(v[4 * j + 3].x, v[4 * j + 3].y, h.w, l.w);
                *reinterpret_cast<uint4 *>(blk + j * kTcLbo) = h;
                *reinterpret_cast<uint4 *>(blk + 1024 + j * kTcLbo) = l;
            }
            fence_proxy_async();
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        tile_sync(g);
        // 3. one thread issues the tile's 12 MMAs (the test hook withholds a unit's: its wait runs out)
        if (rl == 0 && t == 0 && !row_withheld(p, r0)) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            constexpr uint32_t fmt = TCM == MF_FFT_TC_BF16 ? 1u : 0u;
            constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
            const uint32_t a0 = smem_addr(rows_smem + 4 * g * kTcRegion), b0 = smem_addr(Bm);
#pragma unroll
            for (int s = 0; s < 3; ++s) {   // A_hi B_hi, A_hi B_lo, A_lo B_hi
                const uint32_t ab = a0 + (s == 2 ? 1024u : 0u), bb = b0 + (s == 1 ? 8192u : 0u);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t ad = umma_desc(ab + kk * 2 * kTcLbo, kTcLbo, kTcSboA);
                    const uint64_t bd = umma_desc(bb + kk * 2 * kTcLbo, kTcLbo, kTcSboB);
                    const uint32_t acc = (s | kk) != 0 ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&bars[kWarps + g]))
                         : "memory");
        }
        // 4. wait for the products (bounded), read this warp's lanes
        bool mok = true;
        {
            long long it = 0;
            while (!mbar_try_wait_sleep(&bars[kWarps + g], tparity, 1000u)) {
                if (++it > p.spin_limit) { mok = false; break; }
            }
            mok = __all_sync(0xffffffffu, mok);
            tparity ^= 1u;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!mok) {   // the tile stops at the next row's check
            if (t == 0) { atomicOr(p.status, 2); atomicOr(&gfail[g], 1); }
            continue;
        }
        {
            const uint32_t ta = tmem + ((uint32_t)(32 * rl) << 16);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                uint32_t d[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];"
                    : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
                      "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]),
                      "=r"(d[15])
                    : "r"(ta + 16 * c));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    v[8 * c + i] = make_float2(__uint_as_float(d[2 * i]), __uint_as_float(d[2 * i + 1]));
                    if constexpr (TCM == MF_FFT_TC_FP16) v[8 * c + i] = make_float2(v[8 * c + i].x * unscale, v[8 * c + i].y * unscale);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (!has) continue;
        // 5. as the FP32 kernel from the end of stage 0: padded layout, stage 1, epilogue
        const int slot = (int)(r >> p.log2N2);
        const int j2 = (int)(r & (((int64_t)1 << p.log2N2) - 1));
        const int unit = p.unit0 + slot;
        const UnitInfo u = p.units[unit];
#pragma unroll
        for (int q = 0; q < 32; ++q) region[spad(32 * t + q)] = v[q];
        __syncwarp();
        const int64_t rn = r + step;
        GroupRhoSink<L, 1> snk(p, u, j2, region, &bars[w], rn < total ? row_src<L>(p, rn) : nullptr);
        stockham_stage<L, FftShape<L>::R1, 32, +1, true, GroupRhoSink<L, 1>, GroupSync<1>>(region, tw, 0, t, snk);
        snk.finish(&p.partials[((int64_t)unit << p.log2N2) + j2]);
    }
    // every warp is done with tensor memory (a warp that left the loop early
    // issued no tensor-core work after its last completed wait)
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (w == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(2 * kTcCols)
                     : "memory");
    }
}

static size_t rows_smem_tc() {
    return (size_t)kWarps * kTcRegion * sizeof(float2) + (size_t)TwTable<1024>::SIZE * sizeof(float2) + kTcBBytes +
           (kWarps + 2) * sizeof(uint64_t);
}

MF_DEBUG_READER(dbg_read_rows)

bool pass2_rows_applies(int log2N1) { return log2N1 >= 10 && log2N1 <= 12; }

int pass2_rows_partials(int log2N, int log2N2) {   // partials per unit: one per row and warp
    const int lg1 = log2N - log2N2;
    return lg1 > 10 ? (1 << log2N2) << (lg1 - 10) : (1 << log2N2);   // warps per row: N1 / 1024
}

cudaError_t launch_pass2_rows(const SegDev &seg, const UnitInfo *units, int unit0, int n_units, const float2 *exch,
                              float4 *partials, int seg_idx, KeyLayout kl, mf_trigger *staged, uint64_t *keys,
                              unsigned long long *counter, int64_t cap, int *status, long long spin_limit, int n_sm,
                              int fft_mode, int stall_unit, bool peaks_later, cudaStream_t st) {
    if (!pass2_rows_applies(seg.log2N1)) return cudaErrorInvalidValue;
    if (peaks_later && !pass2_rows_peaks_later(seg.log2N1, fft_mode)) return cudaErrorInvalidValue;
    if (fft_mode != MF_FFT_FP32 && seg.log2N1 != 10) return cudaErrorInvalidValue;
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
    p.stall_unit = stall_unit;
    const int64_t rows = (int64_t)n_units << seg.log2N2;
    if (seg.log2N1 == 10) {
        int64_t grid = std::min<int64_t>(2 * (int64_t)n_sm, (rows + kWarps - 1) / kWarps);
        const unsigned gr = (unsigned)std::max<int64_t>(grid, 1);
        if (fft_mode == MF_FFT_TC_FP16)
            k_pass2_rows_tc<MF_FFT_TC_FP16><<<gr, kWarps * 32, rows_smem_tc(), st>>>(p);
        else if (fft_mode == MF_FFT_TC_BF16)
            k_pass2_rows_tc<MF_FFT_TC_BF16><<<gr, kWarps * 32, rows_smem_tc(), st>>>(p);
        else if (peaks_later)
            k_pass2_rows<1024, false><<<gr, kWarps * 32, rows_smem<1024>(), st>>>(p);
        else
            k_pass2_rows<1024, true><<<gr, kWarps * 32, rows_smem<1024>(), st>>>(p);
    } else if (seg.log2N1 == 11) {
        int64_t grid = std::min<int64_t>(2 * (int64_t)n_sm, (rows + kWarps / 2 - 1) / (kWarps / 2));
        const unsigned gr = (unsigned)std::max<int64_t>(grid, 1);
        if (peaks_later) k_pass2_rows_group<2, false><<<gr, kWarps * 32, rows_group_smem<2>(), st>>>(p);
        else k_pass2_rows_group<2, true><<<gr, kWarps * 32, rows_group_smem<2>(), st>>>(p);
    } else {
        int64_t grid = std::min<int64_t>(2 * (int64_t)n_sm, (rows + kWarps / 4 - 1) / (kWarps / 4));
        const unsigned gr = (unsigned)std::max<int64_t>(grid, 1);
        if (peaks_later) k_pass2_rows_group<4, false><<<gr, kWarps * 32, rows_group_smem<4>(), st>>>(p);
        else k_pass2_rows_group<4, true><<<gr, kWarps * 32, rows_group_smem<4>(), st>>>(p);
    }
    return cudaGetLastError();
}

bool pass2_rows_peaks_later(int log2N1, int fft_mode) {
    return log2N1 >= 10 && log2N1 <= 12 && fft_mode == MF_FFT_FP32;
}

cudaError_t launch_peaks_rows(const SegDev &seg, const UnitInfo *units, int unit0, int n_units, int n_all,
                              const float2 *exch, const float4 *partials, int seg_idx, int n_seg, mf_peak *peaks,
                              cudaStream_t st) {
    if (n_units <= 0) return cudaSuccess;
    if (seg.log2N1 == 10) {
        const unsigned grid = (unsigned)((n_units + kWarps - 1) / kWarps);
        k_peaks_rows<<<grid, kWarps * 32, rows_smem<1024>(), st>>>(exch, units, unit0, n_units, n_all, seg.log2N,
                                                                   seg.log2N2, partials, seg_idx, n_seg, peaks);
    } else if (seg.log2N1 == 11) {
        const unsigned grid = (unsigned)((n_units + kWarps / 2 - 1) / (kWarps / 2));
        k_peaks_rows_group<2><<<grid, kWarps * 32, rows_group_smem<2>(), st>>>(
            exch, units, unit0, n_units, n_all, seg.log2N, seg.log2N2, partials, seg_idx, n_seg, peaks);
    } else if (seg.log2N1 == 12) {
        const unsigned grid = (unsigned)((n_units + kWarps / 4 - 1) / (kWarps / 4));
        k_peaks_rows_group<4><<<grid, kWarps * 32, rows_group_smem<4>(), st>>>(
            exch, units, unit0, n_units, n_all, seg.log2N, seg.log2N2, partials, seg_idx, n_seg, peaks);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t rows_kernel_attributes() {
    {
        cudaError_t e0 = init_twiddle_tables();
        if (e0 != cudaSuccess) return e0;
    }
    cudaError_t e = cudaFuncSetAttribute(k_pass2_rows<1024, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)rows_smem<1024>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_pass2_rows<1024, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)rows_smem<1024>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_peaks_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem<1024>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_pass2_rows_tc<MF_FFT_TC_FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)rows_smem_tc());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_pass2_rows_tc<MF_FFT_TC_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)rows_smem_tc());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_pass2_rows_group<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)rows_group_smem<2>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pass2_rows_group<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)rows_group_smem<2>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pass2_rows_group<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)rows_group_smem<4>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pass2_rows_group<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)rows_group_smem<4>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_peaks_rows_group<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)rows_group_smem<2>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_peaks_rows_group<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)rows_group_smem<4>());
    return e;
}

}  // namespace mf
