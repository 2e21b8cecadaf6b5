// mf_pass1.cu -- pass 1 of the bank filter (template generation, weighting
// and column IFFTs, Eq. 1 with the 2PN phase) as a persistent kernel that
// stages the next column tile's inputs in shared memory while the current
// tile is transformed.
//
// The per-tile kernel (k_fft_pass with TemplateSrc / ExchSink) starts every
// tile with its global loads: the band of W for the tile's C columns and one
// anchor record per column row.  Those loads are L2 hits, but all warps of the
// CTA wait on them at once, and with two CTAs per SM (128 registers, 86 KB of
// shared memory each) the other CTA rarely covers the wait.  Here each CTA
// loops over tiles (item = blockIdx.x + i * gridDim.x, template-major) and
// issues cp.async copies of item i + 1's W rows and anchors into a staging
// area right after the column data of item i is in shared memory, so the
// copies run under item i's second Stockham stage and exchange stores.
//
// Shared memory (L <= 1024, two CTAs per SM):
//   column data   C x STRIDE complex64           (as in the per-tile kernel)
//   W staging     L/2 rows x C columns complex64 (32 KB; the upper half of
//                 every column is outside the one-sided spectrum)
//   anchors       L/2 float4 + L/2 float          (one record per row: D >= C)
//   twiddles     the second stage's table w[r * 32 + k] = exp(2 pi i r k / L)
//                 for L <= 512; for L = 1024 (no room for all 32 rows) rows
//                 r <= 16 only, and w[r] = w[r - 16] w[16] for r > 16
//
// Applies to the FP64-anchor phase when the anchor spacing D is at least the
// tile width C and at most N1, for N = 2^16 .. 2^21 (L = 256 .. 1024); every
// other case launches the per-tile kernel.
#include <algorithm>
#include <cstdlib>

#include "mf_filter.cuh"

namespace mf {
namespace {

__device__ __forceinline__ unsigned sh_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sh_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sh_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

struct Pass1PfParams {
    const float2 *W;
    const UnitInfo *units;
    const float4 *anchors;
    const float *anchors4;
    float2 *E;
    int anc_stride, log2D, log2N;
    int unit0, n_items;
};

template <int L, int C>
__host__ __device__ constexpr size_t pf_wbuf_elems() { return (size_t)(L / 2) * C; }

// twiddle entries kept in shared memory (see the layout above)
template <int L>
__host__ __device__ constexpr int pf_tw_elems() { return L == 1024 ? 17 * 32 : TwTable<L>::S1; }

template <int L, int C>
__host__ __device__ constexpr size_t pf_smem_bytes() {
    return pass_data_bytes<L, C>() + pf_wbuf_elems<L, C>() * sizeof(float2) +
           (size_t)(L / 2) * (sizeof(float4) + sizeof(float)) + (size_t)pf_tw_elems<L>() * sizeof(float2);
}

// Issue the copies of one item's inputs: W rows n < L/2 (C consecutive
// columns each, 16-byte chunks, skipped when both columns of a chunk are
// outside the template's band) and the anchor record of every row that has an
// anchor.  Every thread commits one group.
// The band fields of a unit (k_lo, k_hi, g_lo, n_anc: the first 16 bytes of
// its 32-byte-aligned UnitInfo), loaded a full item ahead of their use.
__device__ __forceinline__ int4 pf_band(const Pass1PfParams &p, int slot) {
    return __ldg(reinterpret_cast<const int4 *>(p.units + p.unit0 + slot));
}

template <int L, int C, int LG1>
__device__ __forceinline__ void pf_issue(const Pass1PfParams &p, int item, int4 band, float2 *wbuf, float4 *abuf,
                                         float *abuf4) {
    constexpr int NT = C * (L / 32);
    constexpr int TILES = (1 << LG1) / C;
    constexpr int CH = C / 2;   // 16-byte chunks per row
    const int slot = item / TILES, tile = item - slot * TILES;
    const int k_lo = band.x, k_hi = band.y, g_lo = band.z, n_anc = band.w;
    const int kc = tile * C;
#pragma unroll
    for (int i = 0; i < (L / 2) * CH / NT; ++i) {
        const int c = threadIdx.x + i * NT;
        const int n = c / CH, j = c - n * CH;
        const int k = kc + 2 * j + (n << LG1);
        if (k + 1 >= k_lo && k < k_hi) cp_async16(wbuf + n * C + 2 * j, p.W + k);
    }
    const float4 *anc0 = p.anchors + (int64_t)slot * p.anc_stride;
    const float *anc40 = p.anchors4 + (int64_t)slot * p.anc_stride;
    const int gstep = 1 << (LG1 - p.log2D);
    const int gbase = (kc >> p.log2D) - g_lo;
    for (int n = threadIdx.x; n < L / 2; n += NT) {
        const int a = gbase + n * gstep;
        if (a >= 0 && a < n_anc) {
            cp_async16(abuf + n, anc0 + a);
            cp_async4(abuf4 + n, anc40 + a);
        }
    }
    cp_async_commit();
}

template <int L, int C, int LG1>
__global__ void __launch_bounds__(C *(L / 32), 2) k_pass1_pf(const Pass1PfParams p) {
    using S = FftShape<L>;
    static_assert(S::NST == 2, "two-stage column lengths only");
    constexpr int T = S::T;
    constexpr int NT = C * T;
    constexpr int TILES = (1 << LG1) / C;
    extern __shared__ float2 smem[];
    float2 *wbuf = smem + pass_data_bytes<L, C>() / sizeof(float2);
    float4 *abuf = (float4 *)(wbuf + pf_wbuf_elems<L, C>());
    float *abuf4 = (float *)(abuf + L / 2);
    float2 *tw = (float2 *)(abuf4 + L / 2);
    const int seq = threadIdx.x % C, t = threadIdx.x / C;
    float2 *sq = smem + seq * SeqStride<L, C>::value;
    {   // published by the first item's barrier
        const float2 *src = g_tw_tables + tw_offset<L>();
        for (int m = threadIdx.x; m < pf_tw_elems<L>(); m += NT) tw[m] = __ldg(&src[m]);
    }
    const int D = 1 << p.log2D;
    const typename ExchSink<L, C, +1, LG1>::Params kp{p.E, LG1, p.log2N};

    int item = blockIdx.x;
    int4 band = make_int4(0, 0, 0, 0);
    if (item < p.n_items) {
        band = pf_band(p, item / TILES);
        pf_issue<L, C, LG1>(p, item, band, wbuf, abuf, abuf4);
    }
    for (; item < p.n_items; item += gridDim.x) {
        const int slot = item / TILES, tile = item - slot * TILES;
        const int next = item + (int)gridDim.x;
        const int4 nband = next < p.n_items ? pf_band(p, next / TILES) : make_int4(0, 0, 0, 0);
        const int k_lo = band.x, k_hi = band.y;
        cp_async_wait_all();
        __syncthreads();   // staged inputs visible; the previous item's last stage has read the column data
        float2 v[32];
        {
            const int k1 = tile * C + seq;
            const int k0 = k1 + (t << LG1);
            // offset from the anchor centre, the same on every row (D divides N1)
            const float d = (float)((k1 & (D - 1)) - (D >> 1));
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const int n = t + r * T;
                const int k = k0 + ((r * T) << LG1);
                float2 x = czero();
                if (k >= k_lo && k < k_hi) {
                    const float2 w = wbuf[n * C + seq];
                    const float4 a = abuf[n];
                    const float a4 = abuf4[n];
                    float ph = fmaf(fmaf(fmaf(fmaf(a4, d, a.w), d, a.z), d, a.y), d, a.x);
                    ph -= rintf(ph);
                    float sn, cs;
                    __sincosf(6.283185307179586f * ph, &sn, &cs);
                    x = make_float2(fmaf(w.x, cs, w.y * sn), fmaf(w.y, cs, -w.x * sn));   // W e^{-i 2 pi ph}
                }
                v[r] = x;
            }
        }
        dft32_halfzero<+1>(v);
#pragma unroll
        for (int r = 0; r < 32; ++r) sq[spad(32 * t + r)] = v[r];
        __syncthreads();   // column data complete; every thread has consumed the staged inputs
        if (next < p.n_items) pf_issue<L, C, LG1>(p, next, nband, wbuf, abuf, abuf4);
        ExchSink<L, C, +1, LG1> snk(kp, tile, p.unit0 + slot, slot);
        if constexpr (L == 1024) last_stage_1024_split<+1>(sq, tw, seq, t, snk);
        else stockham_stage<L, S::R1, 32, +1, true>(sq, tw, seq, t, snk);
        band = nband;
    }
}

int g_pf_blocks_per_sm[3] = {0, 0, 0};   // L = 256, 512, 1024
int g_pf_sms = 0;

template <int L>
constexpr int pf_index() { return L == 256 ? 0 : (L == 512 ? 1 : 2); }

struct PfOp {
    const Pass1PfParams *p;
    int n_units;
    cudaStream_t st;
    bool attrs = false;
    template <int N2, int N1>
    cudaError_t run() {
        if constexpr (N2 >= 256 && N2 <= 1024) {
            constexpr int C = seqs_per_cta<N2>(N1);
            constexpr int LG1 = cx_ilog2(N1);
            auto kern = k_pass1_pf<N2, C, LG1>;
            if (attrs) {
                cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)pf_smem_bytes<N2, C>());
                if (e != cudaSuccess) return e;
                int nb = 0;
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, C * (N2 / 32), pf_smem_bytes<N2, C>());
                if (e != cudaSuccess) return e;
                g_pf_blocks_per_sm[pf_index<N2>()] = nb;
                return cudaSuccess;
            }
            Pass1PfParams q = *p;
            q.n_items = n_units * (N1 / C);
            const int per_sm = g_pf_blocks_per_sm[pf_index<N2>()];
            const int grid = (int)std::min<int64_t>(q.n_items, (int64_t)per_sm * g_pf_sms);
            kern<<<grid, C * (N2 / 32), pf_smem_bytes<N2, C>(), st>>>(q);
            return cudaGetLastError();
        } else {
            return cudaErrorNotSupported;
        }
    }
};

}  // namespace

bool pass1_pf_applies(int log2N, int log2D, int phase_mode) {
    if (g_pf_sms <= 0 || phase_mode == MF_PHASE_FP32) return false;
    const char *env = std::getenv("MFGB_P1PF");   // "0": the per-tile kernel (comparisons)
    if (env && env[0] == '0') return false;
    if (log2N < 16 || log2N > 21) return false;
    const int log2N2 = log2_n2(log2N), log2N1 = log2N - log2N2;
    const int C = (8192 >> log2N2) < (1 << log2N1) ? (8192 >> log2N2) : (1 << log2N1);   // seqs_per_cta
    if ((1 << log2D) < C || log2D > log2N1) return false;
    const int idx = log2N2 == 8 ? 0 : (log2N2 == 9 ? 1 : 2);
    return g_pf_blocks_per_sm[idx] >= 1;
}

cudaError_t launch_pass1_pf(const SegDev &seg, const UnitInfo *units, int unit0, int n_units, int log2D,
                            int max_anc, const float4 *anchors, const float *anchors4, float2 *exch,
                            cudaStream_t st) {
    if (n_units <= 0) return cudaSuccess;
    Pass1PfParams p{seg.W, units, anchors, anchors4, exch, max_anc, log2D, seg.log2N, unit0, 0};
    PfOp op{&p, n_units, st};
    return dispatch_split(seg.log2N, op);
}

cudaError_t pass1_pf_kernel_attributes() {
    cudaError_t e = init_twiddle_tables();   // this translation unit's copy of the Stockham tables
    if (e != cudaSuccess) return e;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_pf_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    for (int lg = 16; lg <= 21; ++lg) {
        Pass1PfParams p{};
        PfOp op{&p, 0, nullptr, true};
        if ((e = dispatch_split(lg, op)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace mf
