// mf_internal.h -- structures shared by the host code and the kernels of
// libmfgb (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mfgb.h"

namespace mf {

// G Msun / c^3 in seconds (IAU 2015 nominal solar mass parameter).
constexpr double kMsunS = 4.925490947e-6;
constexpr int kTmplStride = 8;   // doubles per template record

// Per-template constants, FP64, written by mf_bank_create (host):
//   psi(f) = C0 + c1 u + c2 u^2 + c3 u^3 + c5 u^5 in turns (cycles), u = f^(-1/3), f in Hz,
// the 2PN stationary-phase phase Psi/(2 pi) with t_c = phi_c = 0 (C0 = -1/8).
enum TmplField { TF_C1 = 0, TF_C2 = 1, TF_C3 = 2, TF_C5 = 3, TF_FISCO = 4, TF_AMP = 5, TF_M = 6, TF_ETA = 7 };

// Segment constants that kernels read on the device (written by segment prep).
struct SegConsts {
    double P_tot;   // sum_{1 <= k < N/2} f_k^(-7/3) / S_k
    double alpha;   // sqrt(4 df / P_tot): scale of W so that rho is O(1)
};

// What the filter kernels need to know about a segment.
struct SegDev {
    const float2 *W;          // [N/2]  alpha f^(-7/6) conj(s~_k) / S_k, 0 at k = 0
    const double *P;          // [N/2+1] exclusive prefix of f^(-7/3)/S_k
    const SegConsts *consts;  // device
    double fs, df;
    int64_t N;
    int log2N, log2N1, log2N2;   // N = N1 * N2, N2 = column (pass-1) length
    const void *w_tmap = nullptr;   // host copies of two CUtensorMaps over W for pass 1, boxes of C and C/2
                                    // columns (NULL: none)
};

// Per (template, segment) unit, computed on the device for each filter call.
struct UnitInfo {
    int32_t k_lo, k_hi;   // band [k_lo, k_hi)
    int32_t g_lo, n_anc;  // first anchor index and anchor count
    float rho_scale;      // rho = |raw| * rho_scale, raw = sum_band W_k e^{-i Psi_k} e^{2 pi i jk/N}
    float thr2;           // |raw|^2 > thr2  <=>  rho > threshold
    float z_scale;        // z = raw * z_scale (Eq. 1 with A = Mc^(5/6))
    int32_t tmpl;         // template index
};
static_assert(sizeof(UnitInfo) == 32, "the persistent pass 1 reads the band fields as one int4");

// Four-step split N = N1 * N2, N2 the column (pass-1) length: the balanced
// one, N2 = 2^floor(log2 N / 2).
__host__ __device__ inline int log2_n2(int log2N) { return log2N / 2; }

// The filter's alternative split of N = 2^log2N (the autotuner's second
// candidate): column length 2^alt_log2n2, or -1 where there is none.
//   2^18: 256 x 1024 (balanced 512 x 512)     2^19: 1024 x 512 (512 x 1024)
//   2^20: 512 x 2048 (1024 x 1024)            2^21: 2048 x 1024 (1024 x 2048)
//   2^22: 1024 x 4096 (2048 x 2048)
__host__ __device__ inline int alt_log2n2(int log2N) {
    switch (log2N) {
        case 18: return 8;
        case 19: return 10;
        case 20: return 9;
        case 21: return 11;
        case 22: return 10;
        default: return -1;
    }
}

// Anchor slot layout.  A template's G = (N/2)/D anchor groups g (bins
// [g D, g D + D)) are stored column-major over gs = max(1, N1/D) anchor
// columns: g -> (g mod gs) R + g / gs with R = G / gs (= N2/2 when D <= N1).
// A pass-1 column tile (C <= D consecutive columns k1 sharing k1 / D, one
// anchor group per column row n) then reads anchor column k1 / D, rows
// n = 0..N2/2-1, as one contiguous run: record (kc / D) R + n.  With D > N1
// (short segments) gs = 1 and the layout is linear.  A slot holds G records.
__host__ __device__ __forceinline__ int anchor_log2gs(int log2N1, int log2D) {
    return log2N1 > log2D ? log2N1 - log2D : 0;
}
__host__ __device__ __forceinline__ int anchor_log2R(int log2N, int log2N1, int log2D) {
    return log2N - 1 - log2D - anchor_log2gs(log2N1, log2D);
}
__host__ __device__ __forceinline__ int64_t anchor_slot_index(int64_t g, int log2N, int log2N1, int log2D) {
    const int lgs = anchor_log2gs(log2N1, log2D);
    return ((g & ((1 << lgs) - 1)) << anchor_log2R(log2N, log2N1, log2D)) + (g >> lgs);
}
__host__ __device__ __forceinline__ int64_t anchor_slot_records(int log2N, int log2D) {
    return (int64_t)1 << (log2N - 1 - log2D);
}

// Debug builds (nvcc -DMFGB_DEBUG, build.py --debug): the computed indices of
// the exchange stores and loads, the anchor reads and writes, the bulk and TMA
// copies, the row kernels, the persistent queues and the trigger-sort scatter
// are range-checked; a failed check sets its bit in the translation unit's
// status word and the access is skipped.  mf_debug_status reads and clears the
// words.  Release builds compile the checks away.
enum DbgBit : unsigned {
    kDbgExch = 1u,      // exchange index outside the batch slot
    kDbgAnchor = 2u,    // anchor record outside the slot
    kDbgCopy = 4u,      // bulk / TMA copy range outside its source or destination
    kDbgRows = 8u,      // row kernel: row, partial or region index
    kDbgQueue = 16u,    // persistent scheduler: decoded item outside its queue
    kDbgSort = 32u,     // trigger sort: scatter position outside the key count
    kDbgOut = 64u,      // peaks, partials or trigger records outside their arrays
};
#ifdef MFGB_DEBUG
static __device__ unsigned g_dbg_word;
__device__ __forceinline__ bool mf_dbg_ok(bool c, unsigned bit) {
    if (!c) atomicOr(&g_dbg_word, bit);
    return c;
}
#define MF_DBG(cond, bit) mf_dbg_ok((cond), (bit))
#define MF_DEBUG_READER(name)                                                           \
    cudaError_t name(unsigned *w) {                                                     \
        unsigned z = 0;                                                                 \
        cudaError_t e = cudaMemcpyFromSymbol(w, g_dbg_word, sizeof(unsigned));          \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_dbg_word, &z, sizeof(unsigned)); \
        return e;                                                                       \
    }
#else
#define MF_DBG(cond, bit) true
#define MF_DEBUG_READER(name)         \
    cudaError_t name(unsigned *w) {   \
        *w = 0;                       \
        return cudaSuccess;           \
    }
#endif
// the status word of each translation unit that launches kernels
cudaError_t dbg_read_filter(unsigned *w);
cudaError_t dbg_read_pass1(unsigned *w);
cudaError_t dbg_read_rows(unsigned *w);
cudaError_t dbg_read_persist(unsigned *w);
cudaError_t dbg_read_chisq(unsigned *w);
cudaError_t dbg_read_prep(unsigned *w);
cudaError_t dbg_read_fused(unsigned *w);

// Stable trigger keys: (tmpl, seg, j) packed into 64 bits.
struct KeyLayout {
    int j_bits, seg_bits, tmpl_bits;
};

// The persistent scheduler's first queue is a sequence of rounds rho; round
// rho holds, in order, the anchor chunks of unit rho + LA and the pass-1 tiles
// of unit rho (each only if that unit exists).  Rounds with the same
// membership form a regime of equal size.
struct QueueRegime {
    int rho0;      // first round of the regime
    int first;     // queue index of its first item
    int size;      // items per round
    int rounds;    // number of rounds
    int flags;     // 1: anchors, 2: pass 1
};
constexpr int kMaxRegimes = 8;

// Everything the persistent bank scheduler (mf_persist.cu) needs for one segment.
struct PersistParams {
    SegDev seg;
    const double *tmpl;
    const UnitInfo *units;
    QueueRegime reg[kMaxRegimes];   // queue 1: anchor chunks and pass-1 tiles in rounds
    int n_reg;
    int n_items1, n_items2;         // queue 2: pass-2 tiles, unit by unit
    int n_sm, split;                // CTAs with blockIdx mod n_sm < split start on queue 1
    int LA;
    int log2D, max_anc, nA, S, SA;
    float4 *anchors;            // SA slots of max_anc records
    float *anchors4;
    float2 *exch;               // S slots of N complex64
    unsigned *ctl;              // [0] queue-1 head, [1] abort flag, [2] queue-2 head (zeroed before launch)
    unsigned *doneA, *done1, *done2;   // per-unit completed item counts (zeroed before launch)
    int *status;                // bit 1: a bounded wait expired
    float4 *partials;           // [units][pass-2 tiles]
    mf_trigger *staged;
    uint64_t *keys;
    unsigned long long *counter;
    int64_t cap;
    int seg_idx, n_seg;
    KeyLayout kl;
    mf_peak *peaks;
    long long spin_limit;       // bounded-wait iterations (back-off <= ~1 us each)
    int stall_unit;             // test hook: this unit's pass 2 waits for a count never reached (-1: off)
    unsigned long long *stats;  // diagnostics (nullable): per phase [work cycles, wait cycles, items, waited items]
};

// ---- launch wrappers (defined in the .cu files; return cudaError_t) -----

// segment preparation (mf_prep.cu)
cudaError_t launch_forward_fft(const float *s, int64_t N, float2 *exch, float2 *X, cudaStream_t st);
// the same DFT in FP64 (mf_prep64.cu): scratch of N/2 complex128 (8 N bytes), three kernels
cudaError_t launch_forward_fft64(const float *s, int64_t N, void *scratch, float2 *X, cudaStream_t st);
cudaError_t prep64_kernel_attributes();
// batch <= 65535 transforms of N points, x and y batch entries N apart, exch batch * N
cudaError_t launch_fft_c2c(const float2 *x, float2 *y, int64_t N, int batch, int sign, float2 *exch,
                           cudaStream_t st);
cudaError_t launch_psd_weights(const float2 *X, const double *psd, double psd_f0, double psd_S0,
                               int64_t N, double fs, double *q, cudaStream_t st);
cudaError_t launch_prefix_f64(const double *q, int64_t n, double *P, double *block_tmp, cudaStream_t st);
cudaError_t launch_weight_data(const float2 *X, const double *psd, double psd_f0, double psd_S0,
                               int64_t N, double fs, const double *P, SegConsts *consts, float2 *W, float *fac,
                               cudaStream_t st);
cudaError_t launch_apply_weights(const float2 *X, const float *fac, int64_t N, float2 *W, cudaStream_t st);
int64_t prefix_block_tmp_count(int64_t n);

// synthesis (mf_synth.cu)
cudaError_t launch_synth_spectrum(const double *g, int64_t N, double fs, double f_low, const double *psd,
                                  double psd_f0, double psd_S0, const double *inj_dev, int64_t n_inj,
                                  const double *P, double noise_scale, float2 *Y, cudaStream_t st);
cudaError_t launch_inverse_real_fft(const float2 *Y, int64_t N, double scale, float2 *exch, float *s,
                                    cudaStream_t st);

// filter (mf_filter.cu)
// units[i] <- template order[i] (order NULL: template i)
cudaError_t launch_units(const SegDev &seg, const double *tmpl, int n_t, double f_low, float thr,
                         int log2D, const int *order, UnitInfo *units, cudaStream_t st);
cudaError_t launch_anchors(const SegDev &seg, const double *tmpl, const UnitInfo *units, int unit0,
                           int n_units, int log2D, int max_anc, float4 *anchors, float *anchors4,
                           cudaStream_t st, int reps = 1);
// (reps > 1: every record is also stored reps - 1 more times, n_units slots
// apart, for launches that cover several bands of the same templates)
// p1_form: 0 the persistent form with staged inputs (tiles of C columns),
// 1 one CTA per column tile, 2 the persistent form with tiles of C/2 columns
// (the persistent form only where it applies; every form gives bit-identical
// results).  status / spin_limit: the persistent form's bounded wait on its
// input copies (bit 1 of *status on expiry).
cudaError_t launch_pass1(const SegDev &seg, const UnitInfo *units, int unit0, int n_units, int log2D,
                         int max_anc, const float4 *anchors, const float *anchors4, float2 *exch,
                         int phase_mode, const double *tmpl, int p1_form, int *status, long long spin_limit,
                         cudaStream_t st, bool narrow = false);
// narrow: bands of a few rows per column (the chi^2 sub-bands); the staged form
// then starts a column with a cheaper first stage wherever each lane of a warp
// holds at most one row of the band (other forms ignore it; rounding differs
// from the half-zero DFT, within the FP32 error of the transform).
cudaError_t launch_pass2(const SegDev &seg, const UnitInfo *units, int unit0, int n_units,
                         const float2 *exch, float4 *partials, int seg_idx, KeyLayout kl,
                         mf_trigger *staged, uint64_t *keys, unsigned long long *counter, int64_t cap,
                         cudaStream_t st);
int pass2_blocks(int log2N, int log2N2);   // pass-2 tiles per unit for the split N2 = 2^log2N2
// pass 1 as a persistent kernel with cp.async staging of the next tile (mf_pass1.cu);
// launch_pass1 takes it where it applies
bool pass1_pf_applies(int log2N, int log2N2, int log2D, int phase_mode);
cudaError_t launch_pass1_pf(const SegDev &seg, const UnitInfo *units, int unit0, int n_units, int log2D,
                            int max_anc, const float4 *anchors, const float *anchors4, float2 *exch, bool half_tile,
                            int *status, long long spin_limit, cudaStream_t st, bool narrow = false);
// the two tensor maps over W (2 x 128 bytes at maps_out: boxes of C and C/2
// columns) for the persistent pass 1; false if it does not apply (N outside
// 2^16..2^21) or they cannot be made
bool make_w_tensor_maps(const float2 *W, int log2N, int log2N2, void *maps_out);
cudaError_t pass1_pf_kernel_attributes();
// pass 2 with whole rows per warp and bulk-copy prefetch (row length 1024 only)
bool pass2_rows_applies(int log2N1);                 // row length N1 = 2^log2N1
int pass2_rows_partials(int log2N, int log2N2);        // partials per unit: one per row and warp
cudaError_t launch_pass2_rows(const SegDev &seg, const UnitInfo *units, int unit0, int n_units, const float2 *exch,
                              float4 *partials, int seg_idx, KeyLayout kl, mf_trigger *staged, uint64_t *keys,
                              unsigned long long *counter, int64_t cap, int *status, long long spin_limit, int n_sm,
                              int fft_mode, int stall_unit, bool peaks_later, cudaStream_t st);
// peaks_later: 1024-point FP32 rows keep only each row's maximum, and the
// batch's peaks come from launch_peaks_rows (before the exchange is reused)
bool pass2_rows_peaks_later(int log2N1, int fft_mode);
cudaError_t launch_peaks_rows(const SegDev &seg, const UnitInfo *units, int unit0, int n_units, int n_all,
                              const float2 *exch, const float4 *partials, int seg_idx, int n_seg, mf_peak *peaks,
                              cudaStream_t st);
cudaError_t launch_reduce_peaks(const SegDev &seg, const UnitInfo *units, int n_units, const float4 *partials,
                                int nblk, int seg_idx, int n_seg, mf_peak *peaks, cudaStream_t st);
cudaError_t launch_sort_triggers(const unsigned long long *counter, int64_t cap, int key_bits,
                                 const mf_trigger *staged, const uint64_t *keys, uint64_t *keys_tmp,
                                 uint32_t *idx_a, uint32_t *idx_b, uint32_t *ghist, uint64_t *tstat,
                                 unsigned *tickets, mf_trigger *out, uint32_t *perm_out, int64_t *n_out,
                                 int *status, int n_sm, int64_t spin_limit, cudaStream_t st);
int sort_launches(int key_bits);   // kernels queued by launch_sort_triggers
// tile status words the sort needs for cap records (one per 2048-key tile and digit)
inline int64_t sort_tile_words(int64_t cap) { return ((cap + 2047) / 2048) * 256; }

// refinement (mf_refine.cu).  partial: device scratch of refine_scratch_bytes(n, bpr)
// bytes (8 partial sums per block, then one row record of at most kRefRowBytesMax bytes per row)
constexpr size_t kRefRowBytesMax = 128;
size_t refine_scratch_bytes(int64_t n, int bpr);
cudaError_t launch_refine(const SegDev &seg, double f_low, int phase_mode, const double *theta, int64_t n,
                          const int64_t *band, double *obj, double *grad, double *partial, int bpr,
                          cudaStream_t st);
// chi^2 series (Eq. 5): at most this many sub-bands
constexpr int kChisqMaxBands = 64;
cudaError_t launch_chisq_units(const SegDev &seg, const UnitInfo *all, int n_t, const int32_t *tmpl, int n, int p,
                               UnitInfo *out, int64_t *edges, cudaStream_t st);
// mode 0: first sub-band (store |raw|^2), 1: later sub-band (add), 2: full band (write chi^2)
cudaError_t launch_chisq_pass2(const SegDev &seg, const UnitInfo *units, int unit0, int n_units, const float2 *exch,
                               float *acc, int mode, int p, cudaStream_t st);

// trigger clustering scratch (every array sized for the trigger capacity)
struct ClusterScratch {
    uint32_t *flag, *incl, *bsum, *members, *wsum, *rep_count, *idx_a, *idx_b, *perm, *ghist;
    unsigned long long *best;
    mf_trigger *rep, *sorted;
    uint64_t *keys, *keys_tmp, *tstat;
    unsigned *tickets;
    int64_t *n_c, *n_sorted;
    int *status;
};
cudaError_t launch_cluster(const mf_trigger *trig, const int64_t *n_trig, int64_t cap, int window, KeyLayout kl,
                           ClusterScratch &w, mf_event *events, int64_t ev_cap, int64_t *n_events, int n_sm,
                           int64_t spin_limit, cudaStream_t st);
int cluster_launches(int key_bits);
int64_t cluster_scan_blocks(int64_t cap);
cudaError_t launch_chisq_points(const SegDev *segs, int n_seg, const double *tmpl, int n_t, double f_low,
                                int phase_mode, const int32_t *rows, int64_t stride, int64_t n, int p, int bpr,
                                double2 *partial, float *chisq, cudaStream_t st);

// segments of one mf_refine_triggers_multi call (kernel-parameter table)
constexpr int kRefineMaxSegs = 256;
cudaError_t launch_refine_multi(const SegDev *segs, int n_seg, const int32_t *row_seg, double f_low,
                                int phase_mode, const double *theta, int64_t n, const int64_t *band, double *obj,
                                double *grad, double *partial, int bpr, cudaStream_t st);
int refine_blocks_per_row();
int refine_blocks_for(int64_t n, int n_sm);   // blocks per row that fill the GPU
// kernels queued by one refinement call of n rows: the row set-up, the
// partial sums in chunks of at most 65535 rows (grid y limit), the totals
inline int refine_launches(int64_t n) { return 2 + (int)((n + 65534) / 65535); }

// fused persistent scheduler (mf_fused.cu): N = 2^19, 2^20 on the balanced split;
// anchors of all units precomputed (slot u = unit u); ring of S exchange slots;
// ctl[0..2] zeroed, done1 / done2 n_units counters each, zeroed
bool fused_applies(int log2N, int log2N2);
cudaError_t launch_fused(const SegDev &seg, const UnitInfo *units, int n_units, int log2D, int max_anc,
                         const float4 *anchors, const float *anchors4, float2 *ring, int S, double split,
                         unsigned *ctl, unsigned *done1, unsigned *done2, float4 *partials, int seg_idx, KeyLayout kl,
                         mf_trigger *staged, uint64_t *keys, unsigned long long *counter, int64_t cap, int *status,
                         long long spin_limit, int stall_unit, cudaStream_t st);
cudaError_t fused_kernel_attributes();

// persistent scheduler (mf_persist.cu): segments with N >= 2^13
cudaError_t launch_persistent(const PersistParams &P, int grid, cudaStream_t st);
int persist_blocks_per_sm(int log2N);
void persist_tiles(int log2N, int *n1, int *n2);

}  // namespace mf
