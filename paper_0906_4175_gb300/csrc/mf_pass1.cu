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
// starts the copies of item i + 1's W rows and anchors into a staging area
// right after the column data of item i is in shared memory, so the copies
// run under item i's second Stockham stage and exchange stores:
//   W rows      2-D TMA loads (cp.async.bulk.tensor) of the segment's W viewed
//               as [N2/2 rows][N1 columns], boxes of C columns x 64 rows, only
//               the boxes that meet the template's band;
//   anchors     one record per column row: the tile's rows of one anchor
//               column, contiguous in the column-major anchor slot, as two
//               bulk copies (cp.async.bulk) of the rows in the band.
// One thread issues them, completion on an mbarrier (bounded wait).  Without a
// tensor map (segments prepared outside mf_segment_upload), every thread
// copies 16-byte chunks with cp.async instead.
//
// Shared memory (L <= 1024, two CTAs per SM):
//   column data   C x STRIDE complex64           (as in the per-tile kernel)
//   W staging     L/2 rows x C columns complex64 (32 KB; the upper half of
//                 every column is outside the one-sided spectrum)
//   anchors       L/2 float4 + L/2 float          (one record per row: D >= C)
//   twiddles     the second stage's table w[r * 32 + k] = exp(2 pi i r k / L)
//                 for L <= 512; for L = 1024 (no room for all 32 rows) rows
//                 r <= 16 only, and w[r] = w[r - 16] w[16] for r > 16
//   mbarrier      8 bytes
//
// Template generation skips, warp by warp, groups of four column rows that lie
// outside the band of every lane (the rows of a column are 32 N1 bins apart,
// so a template's band covers a contiguous range of them); the arithmetic of
// every in-band bin is that of the per-tile kernel, so results are bit-identical.
//
// Applies to the FP64-anchor phase when the anchor spacing D is at least the
// tile width C and at most N1, for N = 2^16 .. 2^21 and the 1024-point columns
// of the alternative split of 2^22, 4096 rows x 1024 (L = 256 .. 1024); every
// other case launches the per-tile kernel.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "mf_pass1.cuh"

namespace mf {
namespace {

// two CTAs per SM with tiles of C = 8192/L columns (256 threads); three with
// half-width tiles (128 threads, half the column data and W staging)
template <int L, int C, int LG1, bool TMA, bool NARROW = false>
__global__ void __launch_bounds__(C *(L / 32), (C * (L / 32) >= 256) ? 2 : 3)
    k_pass1_pf(const Pass1PfParams p, const __grid_constant__ CUtensorMap wmap) {
    using S = FftShape<L>;
    static_assert(S::NST == 2, "two-stage column lengths only");
    static_assert(pass_data_bytes<L, C>() % 128 == 0, "TMA destinations must be 128-byte aligned");
    constexpr int T = S::T;
    constexpr int NT = C * T;
    constexpr int TILES = (1 << LG1) / C;
    extern __shared__ __align__(128) float2 pf_smem[];
    float2 *wbuf = pf_smem + pass_data_bytes<L, C>() / sizeof(float2);
    float4 *abuf = (float4 *)(wbuf + pf_wbuf_elems<L, C>());
    float *abuf4 = (float *)(abuf + L / 2);
    float2 *tw = (float2 *)(abuf4 + L / 2);
    uint64_t *bar = (uint64_t *)(tw + pf_tw_elems<L>());
    const int seq = threadIdx.x % C, t = threadIdx.x / C;
    float2 *sq = pf_smem + seq * SeqStride<L, C>::value;
    {
        const float2 *src = g_tw_tables + tw_offset<L>();
        for (int m = threadIdx.x; m < pf_tw_elems<L>(); m += NT) tw[m] = __ldg(&src[m]);
    }
    if constexpr (TMA) {
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            mbar_fence_init();
        }
    }
    __syncthreads();   // twiddles and the mbarrier initialised
    const typename ExchSink<L, C, +1, LG1>::Params kp{p.E, LG1, p.log2N};

    int item = blockIdx.x;
    uint32_t parity = 0;
    int4 band = make_int4(0, 0, 0, 0);
    if (item < p.n_items) {
        band = pf_band(p, item / TILES);
        pf_issue<L, C, LG1, TMA>(p, &wmap, item, band, wbuf, abuf, abuf4, bar);
    }
    for (; item < p.n_items; item += gridDim.x) {
        const int slot = item / TILES, tile = item - slot * TILES;
        const int next = item + (int)gridDim.x;
        const int4 nband = next < p.n_items ? pf_band(p, next / TILES) : make_int4(0, 0, 0, 0);
        const int k_lo = band.x, k_hi = band.y;
        bool ok = true;
        if constexpr (TMA) {
            ok = mbar_wait_bounded(bar, parity, p.spin_limit);
            parity ^= 1u;
        }
        if constexpr (!TMA) cp_async_wait_all();
        // staged inputs visible; the previous item's last stage has read the column data
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) atomicOr(p.status, 2);
            return;   // the W copy of this item never completed; no other copy is in flight
        }
        pf_stage1<L, C, LG1, NARROW>(tile, seq, t, k_lo, k_hi, p.log2D, wbuf, abuf, abuf4, sq, tw);
        __syncthreads();   // column data complete; every thread has consumed the staged inputs
        if (next < p.n_items) pf_issue<L, C, LG1, TMA>(p, &wmap, next, nband, wbuf, abuf, abuf4, bar);
        ExchSink<L, C, +1, LG1> snk(kp, tile, p.unit0 + slot, slot);
        if constexpr (L == 1024) last_stage_1024_split<+1>(sq, tw, seq, t, snk);
        else stockham_stage<L, S::R1, 32, +1, true>(sq, tw, seq, t, snk);
        band = nband;
    }
}

// resident CTAs per SM of the persistent form: [L = 256, 512, 1024][tile C, C/2]
int g_pf_blocks_per_sm[3][2] = {{0, 0}, {0, 0}, {0, 0}};
int g_pf_sms = 0;

template <int L>
constexpr int pf_index() { return L == 256 ? 0 : (L == 512 ? 1 : 2); }

template <int N2, int C, int LG1, bool TMA, bool NARROW = false>
cudaError_t pf_attrs(int &nb) {
    constexpr int SM = (int)pf_smem_bytes<N2, C>();
    cudaError_t e =
        cudaFuncSetAttribute(k_pass1_pf<N2, C, LG1, TMA, NARROW>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pass1_pf<N2, C, LG1, TMA, NARROW>, C * (N2 / 32), SM);
    return e;
}

template <int N2, int N1, int C, bool TMA, bool NARROW = false>
cudaError_t pf_launch(const Pass1PfParams &p, const CUtensorMap &map, int n_units, int per_sm, cudaStream_t st) {
    constexpr int LG1 = cx_ilog2(N1);
    Pass1PfParams q = p;
    q.n_items = n_units * (N1 / C);
    const int grid = (int)std::min<int64_t>(q.n_items, (int64_t)per_sm * g_pf_sms);
    k_pass1_pf<N2, C, LG1, TMA, NARROW><<<grid, C * (N2 / 32), pf_smem_bytes<N2, C>(), st>>>(q, map);
    return cudaGetLastError();
}

struct PfOp {
    const Pass1PfParams *p;
    const CUtensorMap *wmaps;   // [2]: boxes of C and C/2 columns; NULL: cp.async staging of W
    int n_units;
    bool half;                  // tiles of C/2 columns (with a tensor map only)
    cudaStream_t st;
    bool attrs = false;
    bool narrow = false;        // narrow bands: the single-row first stage (full tiles with a tensor map, N2 >= 512)
    template <int N2, int N1>
    cudaError_t run() {
        if constexpr (N2 >= 256 && N2 <= 1024) {
            constexpr int C = seqs_per_cta<N2>(N1);
            constexpr int LG1 = cx_ilog2(N1);
            int *nb = g_pf_blocks_per_sm[pf_index<N2>()];
            if (attrs) {
                int a = 0, b = 0, h = 0;
                cudaError_t e = pf_attrs<N2, C, LG1, false>(a);
                if (e == cudaSuccess) e = pf_attrs<N2, C, LG1, true>(b);
                if (e == cudaSuccess) e = pf_attrs<N2, C / 2, LG1, true>(h);
                if constexpr (N2 >= 512) {
                    int d = 0;
                    if (e == cudaSuccess) e = pf_attrs<N2, C, LG1, true, true>(d);
                }
                if (e != cudaSuccess) return e;
                nb[0] = std::min(a, b);
                nb[1] = h;
                return cudaSuccess;
            }
            const char *env = std::getenv("MFGB_P1TMA");   // "0": cp.async staging of W (comparisons)
            if (wmaps != nullptr && !(env && env[0] == '0')) {
                if (half && nb[1] >= 1) return pf_launch<N2, N1, C / 2, true>(*p, wmaps[1], n_units, nb[1], st);
                if constexpr (N2 >= 512) {
                    if (narrow) return pf_launch<N2, N1, C, true, true>(*p, wmaps[0], n_units, nb[0], st);
                }
                return pf_launch<N2, N1, C, true>(*p, wmaps[0], n_units, nb[0], st);
            }
            CUtensorMap none;
            memset(&none, 0, sizeof(none));
            return pf_launch<N2, N1, C, false>(*p, none, n_units, nb[0], st);
        } else {
            return cudaErrorNotSupported;
        }
    }
};

// cuTensorMapEncodeTiled, looked up once through the runtime (no link against
// the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
    }
    return fn;
}

}  // namespace

MF_DEBUG_READER(dbg_read_pass1)

bool pass1_pf_applies(int log2N, int log2N2, int log2D, int phase_mode) {
    if (g_pf_sms <= 0 || phase_mode == MF_PHASE_FP32) return false;
    const char *env = std::getenv("MFGB_P1PF");   // "0": the per-tile kernel (comparisons)
    if (env && env[0] == '0') return false;
    if (log2N < 16 || log2N > 22 || log2N2 < 8 || log2N2 > 10) return false;
    const int log2N1 = log2N - log2N2;
    const int C = (8192 >> log2N2) < (1 << log2N1) ? (8192 >> log2N2) : (1 << log2N1);   // seqs_per_cta
    if ((1 << log2D) < C || log2D > log2N1) return false;
    const int idx = log2N2 == 8 ? 0 : (log2N2 == 9 ? 1 : 2);
    return g_pf_blocks_per_sm[idx][0] >= 1;
}

bool make_w_tensor_maps(const float2 *W, int log2N, int log2N2, void *maps_out) {
    if (log2N < 16 || log2N > 22 || log2N2 < 8 || log2N2 > 10 || W == nullptr || ((uintptr_t)W & 15u) != 0)
        return false;
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const int log2N1 = log2N - log2N2;
    const int C = (8192 >> log2N2) < (1 << log2N1) ? (8192 >> log2N2) : (1 << log2N1);   // seqs_per_cta
    // W[k], k < N/2, as rows n (k = k1 + n N1) of N1 complex64 (8-byte elements)
    const cuuint64_t dims[2] = {(cuuint64_t)1 << log2N1, (cuuint64_t)1 << (log2N2 - 1)};
    const cuuint64_t strides[1] = {(cuuint64_t)sizeof(float2) << log2N1};
    const cuuint32_t estr[2] = {1, 1};
    CUtensorMap *m = (CUtensorMap *)maps_out;
    for (int h = 0; h < 2; ++h) {   // boxes of C and C/2 columns x kBoxRows rows
        const cuuint32_t box[2] = {(cuuint32_t)(C >> h), (cuuint32_t)kBoxRows};
        if (fn(m + h, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, (void *)W, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

cudaError_t launch_pass1_pf(const SegDev &seg, const UnitInfo *units, int unit0, int n_units, int log2D,
                            int max_anc, const float4 *anchors, const float *anchors4, float2 *exch, bool half_tile,
                            int *status, long long spin_limit, cudaStream_t st, bool narrow) {
    if (n_units <= 0) return cudaSuccess;
    Pass1PfParams p{seg.W, units, anchors, anchors4, exch, max_anc, log2D, seg.log2N, unit0, 0, status, spin_limit};
    PfOp op{&p, (const CUtensorMap *)seg.w_tmap, n_units, half_tile, st, false, narrow};
    return dispatch_split2(seg.log2N, seg.log2N2, op);
}

cudaError_t pass1_pf_kernel_attributes() {
    cudaError_t e = init_pass_tables();   // this translation unit's copies of the Stockham tables and four-step roots
    if (e != cudaSuccess) return e;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_pf_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    for (int lg = 16; lg <= 22; ++lg) {   // 2^22: the alternative split only (2048-point columns use k_fft_pass)
        Pass1PfParams p{};
        PfOp op{&p, nullptr, 0, false, nullptr, true};
        if (lg <= 21 && (e = dispatch_split(lg, op)) != cudaSuccess) return e;
        if (alt_log2n2(lg) >= 8 && alt_log2n2(lg) <= 10 && (e = dispatch_split2(lg, alt_log2n2(lg), op)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

}  // namespace mf
