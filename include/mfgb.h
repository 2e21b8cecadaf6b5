/*
 * mfgb.h -- C ABI of libmfgb.so: the frequency-domain matched filter of
 * Chung, Wen, Blair, Cannon & Datta (arXiv:0906.4175) on one GB300 (sm_103a).
 *
 * Equations are numbered in order of appearance in the paper:
 *   (1) z(t) = x(t) + i y(t) = 4 int_0^inf h~_c(f) s~*(f) / S_n(f) e^{2 pi i f t} df
 *   (2) S_n(f), the initial-LIGO noise PSD, f0 = 150 Hz
 *   (3) rho(t) = |z(t)| / sigma
 *   (4) sigma^2 = 4 int_0^inf |h~_c(f)|^2 / S_n(f) df
 * Templates (Sec. 1.1): 2PN stationary-phase phase, Newtonian amplitude,
 * band f_low .. min(Nyquist, f_isco).  The integrals are Riemann sums over the
 * bins k of an N-sample segment: f_k = k df, df = fs/N.
 *
 * Conventions for every entry point:
 *  - Return value: MF_OK (0) or one of the MF_E* codes below; nothing aborts
 *    and nothing throws.  mf_last_error() gives a message for the calling
 *    thread's last failure.
 *  - "device" pointers are CUDA device (or managed) memory on the current
 *    device; "host" pointers are ordinary host memory.  The caller owns every
 *    pointer it passes in; handles own the device memory they allocate and
 *    free it in their destroy call.
 *  - cuda_stream is a cudaStream_t (NULL = the legacy default stream).  Work
 *    is queued on it asynchronously; device outputs are valid once the stream
 *    has synchronised.  Host inputs are consumed before the call returns.
 *  - All kernels are hand-written CUDA for sm_103a; there is no CPU fallback.
 */
#ifndef MFGB_H
#define MFGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MF_OK        0
#define MF_EINVAL    1  /* bad argument: N not a power of two in range, m <= 0, NaN, f_low >= f_cut, ... */
#define MF_ENOMEM    2  /* a device or host allocation failed */
#define MF_ECUDA     3  /* a CUDA runtime call failed (message has the CUDA error string) */
#define MF_EOVERFLOW 4  /* more triggers than trig_cap: the stored ones are a subset, *n_trig is the true count */
#define MF_ETIMEOUT  5  /* a bounded device-side wait ran out; the launch's outputs are invalid */
#define MF_ENOTSUP   6  /* a mode or size this build does not implement */

typedef struct mf_bank_s *mf_bank;
typedef struct mf_segment_s *mf_segment;

/* Template-bank parameters (Sec. 1.1). */
typedef struct {
    double f_low;     /* low-frequency cut-off in Hz (the paper uses 40) */
    int pn_order;     /* phase order in half-PN steps; only 4 (= 2PN, the paper's choice) */
    int amp_order;    /* amplitude order; only 0 (Newtonian, the paper's choice) */
    int phase_mode;   /* MF_PHASE_* below */
    int fft_mode;     /* MF_FFT_* below */
} mf_bank_params;

#define MF_PHASE_ANCHOR 0  /* default: Psi in FP64 at anchor bins, reduced mod 2 pi, FP32 cubic Taylor between them */
#define MF_PHASE_FP64   1  /* Psi in FP64 at every bin (anchor spacing 1) */
#define MF_PHASE_FP32   2  /* Psi in FP32 only, no FP64 reduction (precision-sweep reference; loses accuracy) */
#define MF_FFT_FP32     0  /* default: every FFT stage in FP32 on the CUDA cores */
/* Precision-sweep forms (config "FFT in FP32 vs a tensor-core DFT-GEMM radix stage"): the first radix-32
   stage of the 1024-point rows of pass 2 runs as a tensor-core GEMM (tcgen05.mma, FP32 accumulate in tensor
   memory) on hi + lo 16-bit splits of its inputs and of the DFT matrix (three products: hi*hi + hi*lo +
   lo*hi); everything else stays FP32.  Only segments with N = 2^19 or 2^20 (1024-point rows);
   mf_filter_bank returns MF_ENOTSUP for other N.  chi^2 (mf_chisq_*) always runs in FP32. */
#define MF_FFT_TC_FP16  1  /* FP16 splits (rows scaled by a power of two into the FP16 range) */
#define MF_FFT_TC_BF16  2  /* BF16 splits */

/* Per-(template, segment) peak: the argmax over j of rho_j (lowest j on ties). */
typedef struct {
    float rho;        /* rho at the peak, Eq. (3) */
    int32_t j;        /* sample index of the peak in z (literal Eq. 1: a signal coalescing at
                         sample j0 peaks at j = (N - j0) mod N) */
    float z_re, z_im; /* z_j = x + i y at the peak, Eq. (1), amplitude constant A = Mc^(5/6) */
} mf_peak;

/* One sample with rho_j > threshold. */
typedef struct {
    int32_t tmpl;     /* template index in the bank */
    int32_t seg;      /* index into the segs[] array of the mf_filter_bank call */
    int32_t j;        /* sample index */
    float rho;
    float z_re, z_im;
} mf_trigger;

/* A frequency-domain injection for mf_synth_segment. */
/* An event: a cluster of triggers (mf_cluster_triggers) and its loudest member. */
typedef struct {
    int32_t tmpl;     /* template of the loudest member */
    int32_t seg;      /* segment index */
    int32_t j;        /* sample index of the loudest member */
    float rho;        /* its rho */
    float z_re, z_im; /* its z */
    int32_t n_trig;   /* triggers in the event */
    int32_t n_tmpl;   /* per-template clusters merged into the event */
} mf_event;

typedef struct {
    double m1, m2;    /* component masses, solar masses */
    double snr;       /* optimal SNR the injection is scaled to */
    int64_t j0;       /* time shift in samples: h(t - j0 dt) */
    double phi;       /* constant phase added to the injection */
} mf_injection;

/* Message for the calling thread's last failure ("" if none). */
const char *mf_last_error(void);
/* Library version string. */
const char *mf_version(void);

/* mf_bank_create -- per-template constants for Sec. 1.1's templates.
 * m1, m2: host arrays of n > 0 component masses in solar masses (> 0, finite).
 * params: host; NULL means f_low = 40, 2PN, Newtonian, MF_PHASE_ANCHOR, MF_FFT_FP32.  fft_mode outside
 * MF_FFT_FP32 .. MF_FFT_TC_BF16 returns MF_ENOTSUP.
 * Computes in FP64 on the host the 2PN phase coefficients, f_isco and the
 * amplitude constant of each template and copies them to the device.
 * *out receives the handle (free with mf_bank_destroy).
 * Errors: MF_EINVAL (n <= 0, bad mass, unsupported order), MF_ENOMEM, MF_ECUDA. */
int mf_bank_create(const double *m1, const double *m2, int64_t n,
                   const mf_bank_params *params, mf_bank *out);
int mf_bank_destroy(mf_bank bank);
/* Number of templates (host out). */
int mf_bank_size(mf_bank bank, int64_t *n);

/* Template sharding: templates are independent (Sec. 2, data parallelism
 * over templates and segments), so a bank can be split by template range
 * across processes or devices, each filtering the same segments.
 *
 * mf_bank_partition -- contiguous ranges of near-equal modelled cost:
 * starts[0] = 0 < starts[1] < ... < starts[parts] = n (host int64 array of
 * parts + 1 entries, written), part r being templates [starts[r],
 * starts[r+1]).  The cost of a template is the sum over the n_seg segments
 * (seg_N[s] samples at seg_fs[s] Hz, host arrays) of 16 N + 8 K, the bytes
 * its filter moves (the complex64 exchange written and read, its band of K
 * weighted-data bins, Sec. 1.1 band rule with params->f_low).  Host only, no
 * device work.  Errors: MF_EINVAL (NULL, n <= 0, parts outside [1, n], a bad
 * mass or segment).
 *
 * mf_bank_create_shard -- mf_bank_create for templates [first, first + count)
 * of the n masses m1, m2.  The anchor spacing of the phase evaluation is fixed
 * by all n templates, so the shard filters its templates bit-identically to
 * the bank of all n.  The shard numbers its templates 0 .. count-1 (peaks,
 * triggers): template i of the shard is template first + i of the list.
 * Errors: as mf_bank_create, and MF_EINVAL when the range is not inside [0, n). */
int mf_bank_partition(const double *m1, const double *m2, int64_t n, const mf_bank_params *params,
                      const int64_t *seg_N, const double *seg_fs, int n_seg, int parts, int64_t *starts);
int mf_bank_create_shard(const double *m1, const double *m2, int64_t n, const mf_bank_params *params,
                         int64_t first, int64_t count, mf_bank *out);

/* mf_segment_upload -- data conditioning for Eq. (1), once per segment.
 * s: N float32 samples of s(t) at rate fs (device if s_on_device, else host).
 * N: power of two, 2^10 <= N <= 2^22.  fs > 0.
 * psd: NULL -> Eq. (2) with f0 = psd_f0 and overall scale psd_S0 (the paper
 *      prints no scale; S0 = 1 gives whitened units, rho does not depend on it);
 *      else a host array of N/2+1 FP64 values S_k at f_k = k fs/N (> 0).
 * Queues on cuda_stream: the forward FFT s~_k = dt sum s_n e^{-2 pi i n k/N}
 * (in FP64, each bin then rounded to complex64: the round-off of the transform
 * stays below 1e-16 of the data's total power, so a band far weaker than the
 * data's content outside it, such as detector noise below f_low, keeps FP32
 * precision), the weighting W_k = f_k^(-7/6) conj(s~_k)/S_k (scaled so that
 * rho is O(1) for any PSD scale) and the FP64 prefix table of f^(-7/3)/S_k
 * that gives sigma^2 of Eq. (4) for any band in O(1).  *out owns that device
 * memory.  Errors: MF_EINVAL, MF_ENOMEM, MF_ECUDA. */
int mf_segment_upload(const float *s, int64_t N, double fs, const double *psd,
                      double psd_f0, double psd_S0, int s_on_device, void *cuda_stream,
                      mf_segment *out);
int mf_segment_destroy(mf_segment seg);

/* mf_segment_refresh -- conditions new samples s (N float32, the segment's N,
 * fs and PSD; device if s_on_device, else host) into the existing segment, as
 * mf_segment_upload would, reusing its device memory: a search that walks
 * consecutive segments of one length keeps one handle per stream.  The first
 * call allocates the conditioning scratch (about 12 N bytes) that the segment
 * then keeps; later calls with device samples allocate nothing and queue only
 * kernels on cuda_stream, so they may be captured in a CUDA graph together
 * with mf_filter_bank (the first call must precede the capture).  Work already
 * queued that reads the segment must be ordered before this call (same stream
 * or an event).  Host samples are copied and the stream synchronised before
 * return; they cannot be refreshed inside a capture.
 * Errors: MF_EINVAL (NULL, wrong device, first call or host samples inside a
 * capture), MF_ENOMEM, MF_ECUDA. */
int mf_segment_refresh(mf_segment seg, const float *s, int s_on_device, void *cuda_stream);

/* Precision of the forward FFT in later mf_segment_refresh calls of a
 * segment (mf_segment_upload always uses FP64):
 *   MF_COND_FP64  default: as mf_segment_upload;
 *   MF_COND_FP32  the library's FP32 four-step FFT, about a third of the time,
 *                 with round-off proportional to the data's total power: for
 *                 data whose power outside the band does not dwarf the band's
 *                 (high-passed data).
 * Host only.  Errors: MF_EINVAL (NULL segment, unknown mode). */
#define MF_COND_FP64 0
#define MF_COND_FP32 1
int mf_segment_set_conditioning(mf_segment seg, int mode);
/* Segment length and sample rate (host outs; either may be NULL). */
int mf_segment_info(mf_segment seg, int64_t *N, double *fs);

/* mf_filter_bank -- Eqs. (1), (3), (4) for every (template, segment) pair.
 * For template t and segment s (segs[s]), with the band of Sec. 1.1:
 *   z_j = 4 df sum_band h~_k conj(s~_k)/S_k e^{+2 pi i j k/N},  rho_j = |z_j|/sigma.
 * Writes peaks[t * n_seg + s] (device array of n_templates * n_seg) and every
 * sample with rho_j > threshold to trig (device array of trig_cap records),
 * sorted by (tmpl, seg, j).  *n_trig (device int64) receives the true count,
 * also when it exceeds trig_cap.  Neither h~(f) nor z(t) is stored.
 * segs: host array of n_seg >= 1 handles.  Within a segment the templates
 * are processed widest band first (descending f_isco, ties in bank order:
 * the costliest units start first); outputs are in bank order all the same.
 * The call queues work on
 * cuda_stream and returns; mf_bank_check() reports overflow and device-side
 * timeouts of the last call on this bank.
 * The first call for a given (segment length, bank size, trig_cap) allocates
 * the bank's workspace (mostly the exchange of the templates in flight:
 * min(bank size, 4 GiB / 8N) x 8N bytes by default, the autotuned budget after
 * mf_autotune); later calls allocate nothing and queue only kernels
 * and memsets, so a call may be captured in a CUDA graph once an identical
 * call has run outside the capture (the graph keeps the segment, output and
 * workspace pointers; replays recompute from the segments' current contents).
 * Errors: MF_EINVAL (f_low >= f_cut for some pair, bad sizes, a workspace that
 * would have to grow or stage profiling switched on inside a stream capture),
 * MF_ENOMEM, MF_ECUDA. */
int mf_filter_bank(mf_bank bank, const mf_segment *segs, int n_seg, float threshold,
                   mf_peak *peaks, mf_trigger *trig, int64_t trig_cap, int64_t *n_trig,
                   void *cuda_stream);

/* mf_fft_c2c -- batched complex FP32 FFT with the library's own kernels (the
 * batched transforms the paper timed in Figs. 1-2):
 *   y_b[k] = sum_n x_b[n] exp(sign 2 pi i n k / N),  b < batch, k < N,
 * unnormalised.  x, y: device complex64 (interleaved re, im float pairs,
 * 8-byte aligned), batch entries N apart; y may equal x (in place).
 * N a power of two in [2^10, 2^22]; sign = -1 (forward) or +1.  N = 2^10 and
 * 2^11: one kernel holding whole sequences per CTA, no allocation (capturable).
 * Larger N: the four-step passes through a complex64 exchange of up to 1 GiB
 * allocated on cuda_stream (not capturable), two kernels per 1 GiB of batch.
 * Returns without synchronising.
 * Errors: MF_EINVAL (NULL, size, sign, alignment, N > 2^11 inside a capture),
 * MF_ENOMEM, MF_ECUDA. */
int mf_fft_c2c(const void *x, void *y, int64_t N, int64_t batch, int sign, void *cuda_stream);

/* mf_chisq_series -- the chi^2 consistency test of Eq. (5) (Sec. 1.2) at every
 * sample of one segment, for the bank templates tmpl[0..n) (device int32):
 *   chi^2_j = (p / sigma^2) sum_l |z_l(t_j) - z(t_j)/p|^2,
 * z_l the Eq. (1) sum over sub-band l = [b_l, b_{l+1}) of the template's band,
 * the p sub-bands splitting sigma^2 of Eq. (4) equally: b_0 = k_lo, b_p = k_hi
 * and b_l = the smallest bin k with P[k] - P[k_lo] >= (l/p)(P[k_hi] - P[k_lo]),
 * P the FP64 prefix of |h~|^2/S_n.  In stationary Gaussian noise chi^2 has
 * 2p - 2 degrees of freedom (the paper uses p = 16).
 * chisq: device FP32 [n][N] (row i for template tmpl[i]); edges: NULL or
 * device int64 [n][p+1] receiving b_0..b_p.  A template index outside the
 * bank gives an empty band (a zero row).  1 <= p <= 64, 1 <= n <= 2^24.
 * Cost: p + 1 inverse FFTs of length N per template (at N = 2^19, 2^20 the
 * first passes of a batch's p + 1 bands run as one launch and the second
 * passes as one kernel that sums the sub-bands in registers).
 * Allocates scratch on cuda_stream (p + 1 exchanges of 8 N bytes per
 * template of a batch, batches sized to the bank's exchange budget: 4 GiB
 * unless mf_autotune chose another), so it cannot be captured in a graph, and
 * returns without synchronising.  A bounded device wait that runs out (row
 * copies of the N = 2^19, 2^20 kernel) makes the next mf_bank_check on this
 * bank return MF_ETIMEOUT.
 * Errors: MF_EINVAL (NULL, sizes, devices, f_low >= f_cut, inside a capture),
 * MF_ENOMEM, MF_ECUDA. */
int mf_chisq_series(mf_bank bank, mf_segment seg, const int32_t *tmpl, int64_t n, int p,
                    float *chisq, int64_t *edges, void *cuda_stream);

/* mf_cluster_triggers -- events from triggers (the paper reports events and
 * gives no clustering rule; this is single linkage in time).  trig: device
 * records sorted by (tmpl, seg, j) as mf_filter_bank returns them; *n_trig
 * (device) their count, of which the first min(*n_trig, trig_cap) are read.
 * Pass 1 links the triggers of one (template, segment) whose consecutive
 * samples are at most `window` apart; pass 2 links those clusters' loudest
 * members of all templates of one segment the same way.  Each event is the
 * loudest member (rho; ties: lower j, then lower template).  events: device
 * array of ev_cap records, written sorted by (seg, j); *n_events (device)
 * receives the true event count (compare with ev_cap for truncation).
 * n_tmpl, n_seg, max_N: the bank size, segment count and largest segment
 * length of the filter call (they size the sort keys).  Allocates scratch
 * (about 100 bytes per trigger of trig_cap) on cuda_stream; does not
 * synchronise.
 * Errors: MF_EINVAL (NULL, negative window, sizes), MF_ENOMEM, MF_ECUDA. */
int mf_cluster_triggers(const mf_trigger *trig, const int64_t *n_trig, int64_t trig_cap, int64_t n_tmpl,
                        int n_seg, int64_t max_N, int32_t window, mf_event *events, int64_t ev_cap,
                        int64_t *n_events, void *cuda_stream);

/* mf_chisq_points -- Eq. (5) at single samples: for each row i the template
 * rows[i*stride], segment segs[rows[i*stride+1]] and sample j =
 * rows[i*stride+2] (device int32; stride >= 3 int32 words, so mf_trigger
 * (stride 6) and mf_event (stride 8) arrays can be passed directly),
 *   chisq[i] = (p / sigma^2) sum_l |z_l(t_j) - z(t_j)/p|^2
 * with the sub-bands of mf_chisq_series, evaluated by direct sums over the
 * band (no FFT).  chisq: device float [n]; NaN for a row naming no template,
 * segment or sample.  1 <= p <= 64, 1 <= n_seg <= 256.
 * Errors: MF_EINVAL, MF_ENOMEM, MF_ECUDA. */
int mf_chisq_points(mf_bank bank, const mf_segment *segs, int n_seg, const int32_t *rows, int64_t stride,
                    int64_t n, int p, float *chisq, void *cuda_stream);

/* mf_bank_check -- synchronises cuda_stream, then returns MF_OK, MF_EOVERFLOW
 * (the last mf_filter_bank on this bank found more than trig_cap triggers) or
 * MF_ETIMEOUT (a bounded device-side wait of that call expired). */
int mf_bank_check(mf_bank bank, void *cuda_stream);

/* mf_autotune -- times the candidate schedules of mf_filter_bank for this
 * bank on these segments (the persistent scheduler with 55/60/65% of the SMs
 * starting on template generation + column FFTs; where some segment is
 * N = 2^19 or 2^20, the fused scheduler with 58/60/62% of the SMs on pass 1;
 * and per-batch launches with
 * 512 MiB..8 GiB of exchange in flight, i.e. 64..1024 templates per batch at
 * N = 2^20 and proportionally more at shorter segments, each with the kernel
 * forms of the two passes: pass 1 persistent with the next tile's inputs
 * staged by TMA and bulk copies, in tiles of C = 8192/N2 columns or of C/2
 * (the CTA tile), or one CTA per column tile; pass 2 in warp-owned rows
 * with bulk-copy prefetch, or one CTA per row tile) and keeps the fastest in
 * the bank for later calls (the default is per-batch launches with 4 GiB, the
 * staged pass 1 and the row pass 2 where they apply).  Before those it picks,
 * per segment length N = 2^18 .. 2^22, the four-step split N = N1 x N2 of the
 * per-batch schedule: the balanced one (N2 = 2^floor(log2 N / 2) columns) or
 * an alternative (2^18: 1024 x 256, 2^19: 512 x 1024, 2^20: 2048 x 512,
 * 2^21: 1024 x 2048, 2^22: 4096 x 1024 as N1 x N2), timing each on that
 * length's segments.  It
 * runs each candidate 1 + repeats times on cuda_stream and synchronises; it
 * allocates temporary outputs and may grow the bank's workspace.  threshold
 * should be the one the search will use (it sets the trigger traffic).  If
 * cache_path is not NULL the choice is written there as one JSON line.
 * Results of mf_filter_bank do not depend on the schedule, the kernel forms or
 * the tile (bit-identical); a different split factors the FFT differently, so
 * its results differ by rounding (within the FP32 path's rho bound).  The
 * choice goes to the cache line as "n1_x_n2" per segment length.
 * Errors: MF_EINVAL, MF_ENOMEM, MF_ECUDA. */
int mf_autotune(mf_bank bank, const mf_segment *segs, int n_seg, float threshold, int repeats,
                const char *cache_path, void *cuda_stream);

/* Schedule overrides, read from the environment at every mf_filter_bank call
 * (for comparisons and tests; none but MFGB_SPLIT_ALT changes a result, every
 * other combination is bit-identical):
 *   MFGB_SCHED=batch|persistent|fused
 *                                per-batch launches, the persistent scheduler,
 *                                or the fused scheduler (N = 2^19, 2^20 with
 *                                the FP64-anchor phase and FP32 FFT: after
 *                                one anchor launch, the staged pass 1 and the
 *                                row pass 2 in one launch, exchanging through
 *                                a ring of 64 MiB that stays in L2; other
 *                                segments per batch),
 *                                over the bank's (autotuned) choice
 *   MFGB_BATCH=n                 templates per batch of the per-batch launches
 *   MFGB_SPLIT=x                 fraction of the SMs the persistent scheduler
 *                                starts on queue 1 (anchors + pass 1), or the
 *                                fused scheduler gives to pass 1
 *   MFGB_FUSED_ROLE=cta          the fused scheduler's first CTAs run pass 1
 *                                instead of whole SMs (both CTAs of an SM)
 *   MFGB_P1PF=0                  pass 1 one CTA per column tile instead of the
 *                                persistent kernel with staged inputs
 *   MFGB_P1TILE=half             the persistent pass 1 with tiles of half the
 *                                columns (three CTAs per SM)
 *   MFGB_P1TMA=0                 the persistent pass 1 stages W with per-thread
 *                                cp.async instead of TMA
 *   MFGB_SPLIT_ALT=1|0           per-batch schedule on the alternative split
 *                                of 2^18..2^22 (see mf_autotune) or the
 *                                balanced one (this one changes rounding)
 *   MFGB_P2ROWS=0                pass 2 one CTA per row tile instead of
 *                                warp-owned rows (FP32 FFT form only)
 *   MFGB_UNIT_ORDER=bank         templates in bank order instead of widest
 *                                band first
 *   MFGB_SCHED_STATS=1           the persistent scheduler prints its queue
 *                                wait counts to stderr (synchronises; not
 *                                inside a stream capture) */

/* mf_synth_segment -- seeded synthetic data: stationary Gaussian noise
 * coloured by S_n (Eq. 2, or psd) plus frequency-domain injections, the
 * stand-in for the paper's coloured-noise test data (Sec. 3).
 *   s~_k = noise_scale sqrt(T S_k / 4)(g_{2k} + i g_{2k+1}) for k_lo <= k < N/2
 *          (k_lo = ceil(f_low N/fs): the data are high-passed at f_low),
 *   s~_k += (snr/sigma_i) h~_i,k e^{-2 pi i k j0_i/N} e^{i phi_i} on injection i's band,
 *   s_n = 2 df Re sum_k s~_k e^{+2 pi i n k/N}.
 * g: device array of 2*(N/2) FP64 standard normals.  inj: host array of n_inj
 * records (may be NULL if n_inj = 0).  s_out: device array of N float32.
 * Errors: MF_EINVAL, MF_ENOMEM, MF_ECUDA. */
int mf_synth_segment(const double *g, int64_t N, double fs, double f_low, const double *psd,
                     double psd_f0, double psd_S0, const mf_injection *inj, int64_t n_inj,
                     double noise_scale, float *s_out, void *cuda_stream);

/* mf_refine_triggers -- objective and adjoint for gradient refinement.
 * For each i < n with theta[i] = (m1, m2, t) (device FP64 [n][3], t in
 * seconds) evaluates the Eq. (1) sum directly at continuous t,
 *   z(t) = 4 df sum_band h~_k(m1, m2) conj(s~_k)/S_k e^{2 pi i f_k t},
 * obj[i] = rho^2 = |z(t)|^2 / sigma^2 (Eqs. 3-4) and the analytic gradient
 * grad[i] = d obj / d(m1, m2, t) (device FP64 [n][3]).  The band of each row is
 * band[2i], band[2i+1] (device int64 [n][2], half-open bins) when band is not
 * NULL, else the Sec. 1.1 band at that row's masses; it is held fixed while
 * differentiating.  params: as for mf_bank_create (NULL = defaults).
 * Errors: MF_EINVAL, MF_ENOMEM, MF_ECUDA. */
int mf_refine_triggers(mf_segment seg, const mf_bank_params *params, const double *theta,
                       int64_t n, const int64_t *band, double *obj, double *grad,
                       void *cuda_stream);

/* mf_refine_triggers_multi -- mf_refine_triggers for rows that belong to
 * different segments, in one launch: row i uses segs[row_seg[i]] (row_seg:
 * device int32 [n]; segs: host array of 1 <= n_seg <= 256 handles on the
 * current device).  A row whose row_seg is outside [0, n_seg) gets NaN in
 * obj and grad.  Other arguments, layouts and errors as mf_refine_triggers;
 * a row's result equals that of mf_refine_triggers on its segment up to the
 * grouping of the partial sums (which depends on n). */
int mf_refine_triggers_multi(const mf_segment *segs, int n_seg, const int32_t *row_seg,
                             const mf_bank_params *params, const double *theta, int64_t n,
                             const int64_t *band, double *obj, double *grad, void *cuda_stream);

/* mf_refine_triggers_static -- the same computation as mf_refine_triggers
 * (same arguments; results agree to rounding, as the partial sums are
 * grouped differently) for callers that cannot allocate device
 * memory while they refine: the call makes no cudaMalloc, cudaMallocAsync,
 * cudaFree or other allocating call.  The paper has no counterpart; it exists
 * for ascent loops that run while another component owns the device
 * allocator.  Its per-block partial sums and row records live in one fixed 4.5 MiB array in
 * device global memory that every device which loads the library holds until
 * the process exits; hence n <= 4096 rows per call (larger n returns
 * MF_EINVAL with a message).  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress) and should come before any
 * stream capture on that device.  All calls share the array: two calls whose
 * work overlaps on the GPU (different streams, or different host threads
 * without ordering) race and give wrong results; calls on one stream are
 * ordered and safe.  Nothing in the array needs clearing between calls. */
int mf_refine_triggers_static(mf_segment seg, const mf_bank_params *params, const double *theta,
                              int64_t n, const int64_t *band, double *obj, double *grad,
                              void *cuda_stream);

/* ---- measurement hooks (not part of the paper's method) ------------------ */

/* mf_debug_status -- index checks of a debug build.  A library built with
 * MFGB_DEBUG defined (paper_0906_4175_gb300/build.py --debug) range-checks the
 * computed indices of the exchange stores and loads, the anchor reads and
 * writes, the TMA and bulk copies, the row kernels, the persistent scheduler's
 * decoded items and the trigger sort's scatter; a failed check skips the access
 * and sets a bit: 1 exchange, 2 anchor record, 4 copy range, 8 row kernel,
 * 16 persistent queue item, 32 sort scatter, 64 peaks / partials / trigger
 * record.  Synchronises the device, ORs the bits set since the last call into
 * *word (host) and clears them; *enabled (host, may be NULL) is 1 in a debug
 * build, 0 otherwise (where *word is always 0).  Errors: MF_EINVAL, MF_ECUDA. */
int mf_debug_status(uint32_t *word, int *enabled);

/* Total number of kernels this library has launched in this process (host
 * counter, incremented at every launch on any stream). */
int mf_launch_count(int64_t *n);

/* Stages of mf_filter_bank timed by mf_bank_profile_read. */
#define MF_STAGE_SETUP   0  /* per-unit band / sigma set-up */
#define MF_STAGE_ANCHORS 1  /* FP64 phase anchors */
#define MF_STAGE_PASS1   2  /* template generation + weighting + column IFFTs */
#define MF_STAGE_PASS2   3  /* row IFFTs + rho epilogue */
#define MF_STAGE_FINAL   4  /* peak reduction + trigger sort */
#define MF_STAGE_FUSED   5  /* persistent scheduler (anchors + pass 1 + pass 2 + peaks) or fused (pass 1 + pass 2) in one launch */
#define MF_N_STAGES      6

/* mf_bank_profile -- when on != 0, later mf_filter_bank calls on this bank
 * record a CUDA event pair around every kernel launch (on the call's stream)
 * and the algorithmic bytes each launch moves (band reads, exchange write
 * and read; triggers excluded).  mf_bank_profile_read synchronises the events
 * recorded so far and returns, per stage, the summed device milliseconds,
 * bytes and launch counts (host arrays of MF_N_STAGES), then clears them.
 * Independently of this switch, every public call pushes an NVTX range named
 * after it ("mf_filter_bank", ...) and every stage launch of mf_filter_bank a
 * nested range named after its stage ("setup", "anchors", "pass1", "pass2",
 * "final", "fused"), for profilers that filter on NVTX. */
int mf_bank_profile(mf_bank bank, int on);

/* mf_bank_debug_stall -- test hook for the bounded device-side waits.  With
 * unit >= 0, later mf_filter_bank calls withhold something that template's
 * waits depend on: under the persistent scheduler (N >= 2^13) its row-FFT
 * tiles wait for a completion count that is never reached; in the per-batch
 * rows kernels (N = 2^19 .. 2^22) the bulk copies of its rows are never
 * issued, and in the tensor-core form (fft_mode != MF_FFT_FP32) its tiles'
 * MMAs are never committed; in mf_chisq_series at N = 2^19, 2^20 the row
 * copies of the template list's entry `unit` are never issued.  After spin_limit back-off iterations (each
 * <= ~1 us; <= 0 restores the default of 4e6) the waiting threads give up,
 * set the status, free what they hold (tensor memory) and return, so
 * mf_bank_check then reports MF_ETIMEOUT and the outputs of that call are
 * invalid.  unit < 0 turns the hook off.  Nothing faults: the GPU context
 * stays usable. */
int mf_bank_debug_stall(mf_bank bank, int64_t unit, int64_t spin_limit);

/* mf_debug_fail_alloc -- test hook for the error paths of device allocations
 * (host-side fault injection).  With countdown >= 0, the library's next
 * `countdown` device allocations (cudaMalloc / cudaMallocAsync made by any
 * entry point, on any thread) succeed and the one after fails as if the
 * device were out of memory: that call returns MF_ENOMEM, frees what it had
 * allocated, leaves its handles as they were before the call (a bank's
 * workspace is released and regrown by the next call) and the hook disarms.
 * countdown < 0 disarms it.  Never fails. */
int mf_debug_fail_alloc(int64_t countdown);
int mf_bank_profile_read(mf_bank bank, double *ms, double *bytes, int64_t *launches);

#ifdef __cplusplus
}
#endif
#endif /* MFGB_H */
