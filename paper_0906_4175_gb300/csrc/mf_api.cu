// mf_api.cu -- host side of libmfgb: handles, argument checks, workspace,
// launch schedule, and the extern "C" entry points declared in mfgb.h.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mf_internal.h"
#include "mf_tmpl.cuh"

namespace mf {
cudaError_t filter_kernel_attributes();
cudaError_t prep_kernel_attributes();
// chi^2 of 1024-point rows over all sub-bands in one pass (mf_chisq.cu)
bool chisq_rows_applies(int log2N);
cudaError_t launch_chisq_rows(const SegDev &seg, const float2 *exch, const UnitInfo *full, int unit0, int nb, int p,
                              float *chisq, int *status, long long spin_limit, int stall, int n_sm, cudaStream_t st);
// batched FFT of whole sequences per CTA (mf_prep.cu), N = 1024 and 2048
bool fft_c2c_single_pass(int64_t N);
cudaError_t launch_fft_c2c_single(const float2 *x, float2 *y, int64_t N, int64_t batch, int sign, cudaStream_t st);
cudaError_t synth_kernel_attributes();
cudaError_t refine_kernel_attributes();
cudaError_t chisq_kernel_attributes();
cudaError_t rows_kernel_attributes();
cudaError_t persist_kernel_attributes();
}  // namespace mf

using namespace mf;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

static int set_err(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define MF_CUDA(call)                                                                                  \
    do {                                                                                               \
        cudaError_t _e = (call);                                                                       \
        if (_e != cudaSuccess) {                                                                       \
            if (_e == cudaErrorMemoryAllocation)                                                       \
                return set_err(MF_ENOMEM, "%s: %s (%s:%d)", #call, cudaGetErrorString(_e), __FILE__,  \
                               __LINE__);                                                              \
            return set_err(MF_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(_e), __FILE__,        \
                           __LINE__);                                                                  \
        }                                                                                              \
    } while (0)

extern "C" const char *mf_last_error(void) { return g_err; }

static std::atomic<int64_t> g_launches{0};
static void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
extern "C" int mf_launch_count(int64_t *n) {
    if (!n) return set_err(MF_EINVAL, "NULL argument");
    *n = g_launches.load();
    return MF_OK;
}
extern "C" const char *mf_version(void) { return "mfgb 0.1 (sm_103a)"; }

// One-time per-device kernel attribute set-up (dynamic shared memory > 48 KB).
static int ensure_device_init() {
    static std::mutex mu;
    static std::vector<int> done;
    int dev = 0;
    MF_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(done.begin(), done.end(), dev) != done.end()) return MF_OK;
    MF_CUDA(filter_kernel_attributes());
    MF_CUDA(prep_kernel_attributes());
    MF_CUDA(persist_kernel_attributes());
    MF_CUDA(synth_kernel_attributes());
    MF_CUDA(refine_kernel_attributes());
    MF_CUDA(chisq_kernel_attributes());
    MF_CUDA(rows_kernel_attributes());
    MF_CUDA(pass1_pf_kernel_attributes());
    MF_CUDA(prep64_kernel_attributes());
    MF_CUDA(fused_kernel_attributes());
    done.push_back(dev);
    return MF_OK;
}

static bool is_pow2_in(int64_t N, int lo, int hi) {
    if (N < ((int64_t)1 << lo) || N > ((int64_t)1 << hi)) return false;
    return (N & (N - 1)) == 0;
}

static int ilog2(int64_t n) {
    int r = 0;
    while (((int64_t)1 << (r + 1)) <= n) ++r;
    return r;
}

static int bits_for(int64_t n) {   // bits to hold values 0..n-1
    int b = 0;
    while (((int64_t)1 << b) < n) ++b;
    return b;
}

// |d^n psi / df^n| bound at f from the coefficient magnitudes
static double psi_deriv_bound(const double *rec, double f, int n) {
    const int pw[4] = {1, 2, 3, 5};
    const double c[4] = {rec[TF_C1], rec[TF_C2], rec[TF_C3], rec[TF_C5]};
    double s = 0.0;
    for (int i = 0; i < 4; ++i) {
        const double q = pw[i] / 3.0;
        double fac = 1.0;
        for (int m = 0; m < n; ++m) fac *= (q + m);
        s += fabs(c[i]) * fac * pow(f, -q - n);
    }
    return s;
}

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
// Device allocations of the library go through these two wrappers so that
// mf_debug_fail_alloc can make one of them fail as if the device were out of
// memory (a host-side fault injection for the error paths): after `countdown`
// further allocations succeed, the next one returns cudaErrorMemoryAllocation
// without allocating, and the hook disarms.  -1 = disarmed.
static std::atomic<int64_t> g_fail_alloc{-1};
static bool alloc_fault() {
    int64_t v = g_fail_alloc.load();
    while (v >= 0)
        if (g_fail_alloc.compare_exchange_weak(v, v - 1)) return v == 0;
    return false;
}
template <class T>
static cudaError_t dev_malloc(T **p, size_t bytes) {
    if (alloc_fault()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}
template <class T>
static cudaError_t dev_malloc_async(T **p, size_t bytes, cudaStream_t st) {
    if (alloc_fault()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(p, bytes, st);
}

struct Workspace {
    int64_t exch_elems = 0, n_t = 0, cap = 0, anc_elems = 0, nblk = 0;
    UnitInfo *units = nullptr;
    float2 *exch = nullptr;
    float4 *anchors = nullptr;
    float *anchors4 = nullptr;
    float4 *partials = nullptr;
    mf_trigger *staged = nullptr;
    uint64_t *keys = nullptr, *keys_tmp = nullptr;
    uint32_t *idx_a = nullptr, *idx_b = nullptr;
    uint32_t *ghist = nullptr;    // trigger sort: digit histograms of every pass
    uint64_t *tstat = nullptr;    // trigger sort: look-back status per (tile, digit)
    unsigned *tickets = nullptr;  // trigger sort: tile tickets per pass
    unsigned long long *counter = nullptr;
    int *status = nullptr;
    unsigned *ctl = nullptr;      // persistent scheduler: [1] abort, then doneA, done1, done2 per unit
    void release() {
        cudaFree(units); cudaFree(exch); cudaFree(anchors); cudaFree(anchors4); cudaFree(partials);
        cudaFree(staged); cudaFree(keys); cudaFree(keys_tmp); cudaFree(idx_a); cudaFree(idx_b);
        cudaFree(ghist); cudaFree(tstat); cudaFree(tickets);
        cudaFree(counter); cudaFree(status); cudaFree(ctl);
        *this = Workspace();
    }
};

struct ProfRec {
    int stage;
    cudaEvent_t a, b;
    double bytes;
};

struct mf_bank_s {
    int64_t n = 0;
    mf_bank_params params{};
    double *d_tmpl = nullptr;
    std::vector<double> fisco;   // host copy of f_isco per template (profiling byte counts)
    // unit order of every segment: descending cost.  A template's band runs
    // from f_low to min(f_isco, fs/2), so descending f_isco (ties in bank
    // order) puts the widest bands first for every segment.  pos is the inverse.
    std::vector<int> order, pos;
    int *d_order = nullptr;
    double B1 = 0.0, B5 = 0.0, fisco_min = 0.0;
    int device = 0;
    Workspace ws;
    bool prof_on = false;
    std::vector<ProfRec> prof;
    cudaStream_t side = nullptr;      // anchors of the next batch run here, beside pass 2
    cudaEvent_t ev_p1 = nullptr, ev_anc = nullptr;
    int64_t stall_unit = -1;          // test hook (mf_bank_debug_stall)
    long long spin_limit = 4000000;   // bounded-wait iterations, back-off <= ~1 us each
    // schedule (defaults until mf_autotune measures this bank): 0 = persistent
    // scheduler, 1 = per-batch launches, 2 = fused scheduler (N = 2^19, 2^20;
    // other lengths per batch); exchange bytes in flight per batch
    // (templates per batch = tuned_exch / (8 N), 0 = the default budget);
    // fraction of SMs that start on queue 1
    int sched = 1;
    int64_t tuned_exch = 0;
    double split = 0.60;
    // kernel forms of the per-batch schedule: pass 1 persistent with staged
    // inputs (0), per tile (1), or persistent with tiles of half the width (2);
    // pass 2 in warp-owned rows (0) or per tile (1)
    int p1_kind = 0, p2_kind = 0;
    // per segment length 2^i: the per-batch schedule uses the alternative
    // split N = N1 * N2 (alt_log2n2) instead of the balanced one
    unsigned char alt_split[23] = {0};
    int *chi_status = nullptr;        // status of the last mf_chisq_series (bit 2: a bounded wait ran out)
};

// Records an event before a launch when profiling; returns the record index or -1.
// NVTX ranges: one per public call and one per stage launch of mf_filter_bank
// (host-side markers a profiler can filter on, e.g. ncu --nvtx --nvtx-include
// "mf_filter_bank/pass1/"; without a profiler attached they cost a call).
struct NvtxRange {
    int level;   // nesting level of this range (negative when no tool tracks ranges)
    explicit NvtxRange(const char *name) : level(nvtxRangePushA(name)) {}
    ~NvtxRange() {   // also ends a stage range that an error return left open
        while (nvtxRangePop() > level) {
        }
    }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
static const char *const kStageNames[MF_N_STAGES] = {"setup", "anchors", "pass1", "pass2", "final", "fused"};

static int prof_begin(mf_bank_s *b, int stage, double bytes, cudaStream_t st) {
    nvtxRangePushA(stage >= 0 && stage < MF_N_STAGES ? kStageNames[stage] : "stage");   // popped by prof_end
    if (!b->prof_on) return -1;
    ProfRec r;
    r.stage = stage;
    r.bytes = bytes;
    if (cudaEventCreate(&r.a) != cudaSuccess) return -1;
    if (cudaEventCreate(&r.b) != cudaSuccess) { cudaEventDestroy(r.a); return -1; }
    cudaEventRecord(r.a, st);
    b->prof.push_back(r);
    return (int)b->prof.size() - 1;
}
static void prof_end(mf_bank_s *b, int idx, cudaStream_t st) {
    if (idx >= 0) cudaEventRecord(b->prof[idx].b, st);
    nvtxRangePop();
}

struct mf_segment_s {
    int64_t N = 0;
    double fs = 0.0;
    int log2N = 0;
    float2 *W = nullptr;
    double *P = nullptr;
    SegConsts *consts = nullptr;
    int device = 0;
    // kept for mf_segment_refresh: the PSD (device copy of a table, or the
    // Eq. (2) parameters) and, after the first refresh, conditioning scratch
    double *psd = nullptr;
    double psd_f0 = 0.0, psd_S0 = 0.0;
    float *fac = nullptr;          // a_k = alpha f^(-7/6) dt / S_k: W_k = a_k conj(X_k) for new samples
    float2 *r_exch = nullptr, *r_X = nullptr;
    float *r_s = nullptr;
    int cond = MF_COND_FP64;       // precision of the forward DFT in mf_segment_refresh
    // CUtensorMaps over W for pass 1 (boxes of C and C/2 columns), for the
    // balanced split [0] and the alternative one [1] (valid when has_tmap[i])
    alignas(64) unsigned char w_tmap[2][256];
    bool has_tmap[2] = {false, false};
    void release() {
        cudaFree(W); cudaFree(P); cudaFree(consts); cudaFree(psd); cudaFree(fac);
        cudaFree(r_exch); cudaFree(r_X); cudaFree(r_s);
        W = nullptr; P = nullptr; consts = nullptr; psd = nullptr; fac = nullptr;
        r_exch = nullptr; r_X = nullptr; r_s = nullptr;
    }
};

static bool stream_capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
    return cs != cudaStreamCaptureStatusNone;
}

static mf_bank_params default_params() {
    mf_bank_params p;
    p.f_low = 40.0;
    p.pn_order = 4;
    p.amp_order = 0;
    p.phase_mode = MF_PHASE_ANCHOR;
    p.fft_mode = MF_FFT_FP32;
    return p;
}

static int check_params(const mf_bank_params &p) {
    if (!(p.f_low > 0.0) || !isfinite(p.f_low)) return set_err(MF_EINVAL, "f_low must be > 0 and finite");
    if (p.pn_order != 4) return set_err(MF_ENOTSUP, "pn_order %d: only 4 (2PN) is implemented", p.pn_order);
    if (p.amp_order != 0) return set_err(MF_ENOTSUP, "amp_order %d: only 0 (Newtonian) is implemented", p.amp_order);
    if (p.phase_mode < 0 || p.phase_mode > 2) return set_err(MF_EINVAL, "phase_mode %d", p.phase_mode);
    if (p.fft_mode < MF_FFT_FP32 || p.fft_mode > MF_FFT_TC_BF16)
        return set_err(MF_ENOTSUP, "fft_mode %d: MF_FFT_FP32, MF_FFT_TC_FP16 or MF_FFT_TC_BF16", p.fft_mode);
    return MF_OK;
}

// A bank of templates [first, first + count) of the mass list m1, m2 (n
// entries).  The phase-derivative bounds that fix the anchor spacing are taken
// over all n templates, so every shard of a list uses the spacing the whole
// list would and filters its templates exactly as the whole bank does.
static int bank_create_range(const double *m1, const double *m2, int64_t n, const mf_bank_params *params,
                             int64_t first, int64_t count, mf_bank *out) {
    if (!out) return set_err(MF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!m1 || !m2 || n <= 0) return set_err(MF_EINVAL, "need n > 0 masses");
    if (first < 0 || count <= 0 || first > n - count)
        return set_err(MF_EINVAL, "templates [%lld, %lld) outside the %lld masses", (long long)first,
                       (long long)(first + count), (long long)n);
    if (count > (int64_t)1 << 24) return set_err(MF_EINVAL, "at most 2^24 templates per bank");
    mf_bank_params p = params ? *params : default_params();
    int rc = check_params(p);
    if (rc) return rc;
    int r0 = ensure_device_init();
    if (r0) return r0;
    std::vector<double> rec((size_t)count * kTmplStride);
    double B1 = 0.0, B5 = 0.0, fmin = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        if (!(m1[i] > 0.0) || !(m2[i] > 0.0) || !isfinite(m1[i]) || !isfinite(m2[i]))
            return set_err(MF_EINVAL, "template %lld: masses must be finite and > 0", (long long)i);
        double tmp[kTmplStride];
        const bool mine = i >= first && i < first + count;
        double *r = mine ? &rec[(size_t)(i - first) * kTmplStride] : tmp;
        template_constants(m1[i], m2[i], r);
        B1 = std::max(B1, psi_deriv_bound(r, p.f_low, 1));
        B5 = std::max(B5, psi_deriv_bound(r, p.f_low, 5));
        if (mine) fmin = std::min(fmin, r[TF_FISCO]);
    }
    n = count;
    mf_bank b = new (std::nothrow) mf_bank_s();
    if (!b) return set_err(MF_ENOMEM, "host allocation");
    b->n = n;
    b->params = p;
    b->B1 = B1;
    b->B5 = B5;
    b->fisco_min = fmin;
    b->fisco.resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) b->fisco[(size_t)i] = rec[(size_t)i * kTmplStride + TF_FISCO];
    b->order.resize((size_t)n);
    b->pos.resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) b->order[(size_t)i] = (int)i;
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](int x, int y) { return b->fisco[(size_t)x] > b->fisco[(size_t)y]; });
    for (int64_t i = 0; i < n; ++i) b->pos[(size_t)b->order[(size_t)i]] = (int)i;
    cudaGetDevice(&b->device);
    cudaError_t e = dev_malloc(&b->d_tmpl, sizeof(double) * rec.size());
    if (e == cudaSuccess) e = cudaMemcpy(b->d_tmpl, rec.data(), sizeof(double) * rec.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = dev_malloc(&b->d_order, sizeof(int) * (size_t)n);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_order, b->order.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(b->d_tmpl);
        cudaFree(b->d_order);
        delete b;
        return set_err(e == cudaErrorMemoryAllocation ? MF_ENOMEM : MF_ECUDA, "bank upload: %s",
                       cudaGetErrorString(e));
    }
    *out = b;
    return MF_OK;
}

extern "C" int mf_bank_create(const double *m1, const double *m2, int64_t n, const mf_bank_params *params,
                              mf_bank *out) {
    return bank_create_range(m1, m2, n, params, 0, n, out);
}

extern "C" int mf_bank_create_shard(const double *m1, const double *m2, int64_t n, const mf_bank_params *params,
                                    int64_t first, int64_t count, mf_bank *out) {
    return bank_create_range(m1, m2, n, params, first, count, out);
}

// Contiguous template ranges of near-equal modelled cost: per template
// sum over segments of 16 N (the exchange written and read) + 8 K (its band
// of W), with K from the Sec. 1.1 band rule.
extern "C" int mf_bank_partition(const double *m1, const double *m2, int64_t n, const mf_bank_params *params,
                                 const int64_t *seg_N, const double *seg_fs, int n_seg, int parts,
                                 int64_t *starts) {
    if (!m1 || !m2 || !seg_N || !seg_fs || !starts) return set_err(MF_EINVAL, "NULL argument");
    if (n <= 0 || n_seg < 1 || parts < 1) return set_err(MF_EINVAL, "need n > 0, n_seg >= 1, parts >= 1");
    if (parts > n) return set_err(MF_EINVAL, "%d parts for %lld templates", parts, (long long)n);
    mf_bank_params p = params ? *params : default_params();
    int rc = check_params(p);
    if (rc) return rc;
    for (int s = 0; s < n_seg; ++s)
        if (seg_N[s] < 2 || !(seg_fs[s] > 0.0)) return set_err(MF_EINVAL, "segment %d: bad N or fs", s);
    std::vector<double> prefix((size_t)n + 1, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        if (!(m1[i] > 0.0) || !(m2[i] > 0.0) || !isfinite(m1[i]) || !isfinite(m2[i]))
            return set_err(MF_EINVAL, "template %lld: masses must be finite and > 0", (long long)i);
        double r[kTmplStride];
        template_constants(m1[i], m2[i], r);
        double c = 0.0;
        for (int s = 0; s < n_seg; ++s) {
            const double N = (double)seg_N[s], fs = seg_fs[s];
            const double fc = std::min(r[TF_FISCO], 0.5 * fs);
            const int64_t lo = std::max((int64_t)1, (int64_t)ceil(p.f_low * N / fs));
            const int64_t hi = std::min((int64_t)floor(fc * N / fs) + 1, seg_N[s] / 2);
            c += 16.0 * N + 8.0 * (double)std::max<int64_t>(0, hi - lo);
        }
        prefix[(size_t)i + 1] = prefix[(size_t)i] + c;
    }
    const double total = prefix[(size_t)n];
    starts[0] = 0;
    for (int r = 1; r < parts; ++r) {
        const double target = total * (double)r / (double)parts;
        int64_t i = std::lower_bound(prefix.begin(), prefix.end(), target) - prefix.begin();
        if (i > 0 && target - prefix[(size_t)i - 1] < prefix[(size_t)i] - target) --i;   // nearer boundary
        const int64_t lo = starts[r - 1] + 1, hi = n - (parts - r);   // every part non-empty
        starts[r] = std::min(std::max(i, lo), hi);
    }
    starts[parts] = n;
    return MF_OK;
}

extern "C" int mf_bank_destroy(mf_bank b) {
    if (!b) return MF_OK;
    for (auto &r : b->prof) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    b->ws.release();
    cudaFree(b->d_tmpl);
    cudaFree(b->d_order);
    cudaFree(b->chi_status);
    if (b->ev_p1) cudaEventDestroy(b->ev_p1);
    if (b->ev_anc) cudaEventDestroy(b->ev_anc);
    if (b->side) cudaStreamDestroy(b->side);
    delete b;
    return MF_OK;
}

extern "C" int mf_bank_size(mf_bank b, int64_t *n) {
    if (!b || !n) return set_err(MF_EINVAL, "NULL argument");
    *n = b->n;
    return MF_OK;
}

// ---------------------------------------------------------------------------
// segments
// ---------------------------------------------------------------------------
extern "C" int mf_segment_upload(const float *s, int64_t N, double fs, const double *psd, double psd_f0,
                                 double psd_S0, int s_on_device, void *cuda_stream, mf_segment *out) {
    NvtxRange nvtx("mf_segment_upload");
    if (!out) return set_err(MF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!s) return set_err(MF_EINVAL, "s is NULL");
    if (!is_pow2_in(N, 10, 22)) return set_err(MF_EINVAL, "N = %lld must be a power of two in [2^10, 2^22]", (long long)N);
    if (!(fs > 0.0) || !isfinite(fs)) return set_err(MF_EINVAL, "fs must be > 0");
    if (!psd && (!(psd_f0 > 0.0) || !(psd_S0 > 0.0) || !isfinite(psd_f0) || !isfinite(psd_S0)))
        return set_err(MF_EINVAL, "psd_f0 and psd_S0 must be > 0");
    int r0 = ensure_device_init();
    if (r0) return r0;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int64_t half = N / 2;
    mf_segment g = new (std::nothrow) mf_segment_s();
    if (!g) return set_err(MF_ENOMEM, "host allocation");
    g->N = N;
    g->fs = fs;
    g->log2N = ilog2(N);
    g->psd_f0 = psd_f0;
    g->psd_S0 = psd_S0;
    cudaGetDevice(&g->device);
    float *s_dev = nullptr;
    float2 *exch = nullptr, *X = nullptr;
    double *q = nullptr, *btmp = nullptr, *psd_dev = nullptr;
    const int64_t nbt = prefix_block_tmp_count(half);
    cudaError_t e = dev_malloc(&g->W, sizeof(float2) * half);
    if (e == cudaSuccess) {   // pass 1's TMA views of W, both splits
        g->has_tmap[0] = make_w_tensor_maps(g->W, g->log2N, log2_n2(g->log2N), g->w_tmap[0]);
        g->has_tmap[1] = alt_log2n2(g->log2N) > 0 && make_w_tensor_maps(g->W, g->log2N, alt_log2n2(g->log2N), g->w_tmap[1]);
    }
    if (e == cudaSuccess) e = dev_malloc(&g->fac, sizeof(float) * half);
    if (e == cudaSuccess) e = dev_malloc(&g->P, sizeof(double) * (half + 1));
    if (e == cudaSuccess) e = dev_malloc(&g->consts, sizeof(SegConsts));
    if (e == cudaSuccess) e = dev_malloc_async(&exch, sizeof(float2) * N, st);
    if (e == cudaSuccess) e = dev_malloc_async(&X, sizeof(float2) * (half + 1), st);
    if (e == cudaSuccess) e = dev_malloc_async(&q, sizeof(double) * half, st);
    if (e == cudaSuccess) e = dev_malloc_async(&btmp, sizeof(double) * nbt, st);
    if (e == cudaSuccess && !s_on_device) {
        e = dev_malloc_async(&s_dev, sizeof(float) * N, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s_dev, s, sizeof(float) * N, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess && psd) {   // kept by the segment for mf_segment_refresh
        e = dev_malloc(&g->psd, sizeof(double) * (half + 1));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g->psd, psd, sizeof(double) * (half + 1), cudaMemcpyHostToDevice, st);
        psd_dev = g->psd;
    }
    const float *s_use = s_on_device ? s : s_dev;
    if (e == cudaSuccess) e = launch_forward_fft64(s_use, N, exch, X, st);   // exch: 8 N bytes = N/2 complex128
    if (e == cudaSuccess) e = launch_psd_weights(X, psd_dev, psd_f0, psd_S0, N, fs, q, st);
    if (e == cudaSuccess) e = launch_prefix_f64(q, half, g->P, btmp, st);
    if (e == cudaSuccess) e = launch_weight_data(X, psd_dev, psd_f0, psd_S0, N, fs, g->P, g->consts, g->W, g->fac, st);
    if (e == cudaSuccess) count_launches(8);   // 3 FFT kernels, weights, 3 scan kernels, weighting
    if (s_dev) cudaFreeAsync(s_dev, st);
    if (exch) cudaFreeAsync(exch, st);
    if (X) cudaFreeAsync(X, st);
    if (q) cudaFreeAsync(q, st);
    if (btmp) cudaFreeAsync(btmp, st);
    if (e == cudaSuccess && !s_on_device) e = cudaStreamSynchronize(st);   // host s / psd consumed before return
    else if (e == cudaSuccess && psd) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        g->release();
        delete g;
        return set_err(e == cudaErrorMemoryAllocation ? MF_ENOMEM : MF_ECUDA, "segment_upload: %s",
                       cudaGetErrorString(e));
    }
    *out = g;
    return MF_OK;
}

extern "C" int mf_segment_refresh(mf_segment g, const float *s, int s_on_device, void *cuda_stream) {
    NvtxRange nvtx("mf_segment_refresh");
    if (!g || !s) return set_err(MF_EINVAL, "NULL argument");
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != g->device) return set_err(MF_EINVAL, "segment lives on device %d, current is %d", g->device, cur);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const bool capturing = stream_capturing(st);
    const int64_t N = g->N, half = N / 2;
    if (!g->r_exch) {
        if (capturing) return set_err(MF_EINVAL, "the first mf_segment_refresh of a segment must precede stream capture");
        cudaError_t e = dev_malloc(&g->r_exch, sizeof(float2) * N);
        if (e == cudaSuccess) e = dev_malloc(&g->r_X, sizeof(float2) * (half + 1));
        if (e != cudaSuccess) {
            cudaFree(g->r_exch); cudaFree(g->r_X);
            g->r_exch = nullptr; g->r_X = nullptr;
            return set_err(e == cudaErrorMemoryAllocation ? MF_ENOMEM : MF_ECUDA, "segment_refresh: %s",
                           cudaGetErrorString(e));
        }
    }
    const float *s_use = s;
    if (!s_on_device) {
        if (capturing) return set_err(MF_EINVAL, "host samples cannot be refreshed inside a stream capture");
        if (!g->r_s) MF_CUDA(dev_malloc(&g->r_s, sizeof(float) * N));
        MF_CUDA(cudaMemcpyAsync(g->r_s, s, sizeof(float) * N, cudaMemcpyHostToDevice, st));
        s_use = g->r_s;
    }
    // the PSD and with it P, sigma's normalisation and the factors a_k are unchanged
    if (g->cond == MF_COND_FP32) {
        MF_CUDA(launch_forward_fft(s_use, N, g->r_exch, g->r_X, st));
        count_launches(2);
    } else {
        MF_CUDA(launch_forward_fft64(s_use, N, g->r_exch, g->r_X, st));
        count_launches(3);
    }
    MF_CUDA(launch_apply_weights(g->r_X, g->fac, N, g->W, st));
    count_launches(1);
    if (!s_on_device) MF_CUDA(cudaStreamSynchronize(st));   // host s consumed before return
    return MF_OK;
}

extern "C" int mf_segment_set_conditioning(mf_segment g, int mode) {
    if (!g) return set_err(MF_EINVAL, "NULL segment");
    if (mode != MF_COND_FP64 && mode != MF_COND_FP32) return set_err(MF_EINVAL, "unknown conditioning mode %d", mode);
    g->cond = mode;
    return MF_OK;
}

extern "C" int mf_segment_destroy(mf_segment g) {
    if (!g) return MF_OK;
    g->release();
    delete g;
    return MF_OK;
}

extern "C" int mf_segment_info(mf_segment g, int64_t *N, double *fs) {
    if (!g) return set_err(MF_EINVAL, "NULL segment");
    if (N) *N = g->N;
    if (fs) *fs = g->fs;
    return MF_OK;
}

// The segment as the kernels see it, with the split N = N1 * N2 (N2 =
// 2^log2N2: the balanced split by default, or the alternative one).
static SegDev seg_dev(const mf_segment_s *g, int log2N2 = -1) {
    SegDev d;
    d.W = g->W;
    d.P = g->P;
    d.consts = g->consts;
    d.fs = g->fs;
    d.df = g->fs / (double)g->N;
    d.N = g->N;
    d.log2N = g->log2N;
    const int alt = (log2N2 >= 0 && log2N2 != log2_n2(g->log2N) && log2N2 == alt_log2n2(g->log2N)) ? 1 : 0;
    d.log2N2 = alt ? log2N2 : log2_n2(g->log2N);
    d.log2N1 = g->log2N - d.log2N2;
    d.w_tmap = g->has_tmap[alt] ? (const void *)g->w_tmap[alt] : nullptr;
    return d;
}

// Anchor spacing D = 2^log2D for a (bank, segment): the largest power of two
// (<= 256) for which the quartic-Taylor remainder max|d^5 psi/dk^5| (D/2)^5/120
// stays below 5e-7 turns and |d psi/dk| D/2 below 16 turns (FP32 magnitude of
// the Taylor sum), both bounded at f_low over the whole bank (k-derivatives are
// f-derivatives times df^n).
static int choose_log2D(const mf_bank_s *b, const mf_segment_s *g) {
    if (b->params.phase_mode == MF_PHASE_FP64) return 0;
    return anchor_log2D(b->B1, b->B5, g->fs / (double)g->N);
}

// templates in flight per batch (exchange ring of batch * N complex64)
// Default exchange budget of the per-batch launches: 4 GiB (512 templates in
// flight at N = 2^20).  Fewer, longer launches leave fewer partly idle tails
// (bench workload: 1 GiB 247k, 2 GiB 250k, 4 GiB 252k, 8 GiB 253k
// templates/s; the chi^2 series at p = 16: 1 GiB 13.3k, 4 GiB 14.4k
// templates/s); mf_autotune replaces it per bank.  mf_fft_c2c, which
// allocates its exchange per call, keeps 1 GiB.
constexpr int64_t kExchBudget = (int64_t)4 << 30;
constexpr int64_t kScratchBudget = (int64_t)1 << 30;

static int64_t choose_batch(int64_t N, int64_t n_t, int64_t tuned_exch) {
    int64_t b = (tuned_exch > 0 ? tuned_exch : kExchBudget) / (8 * N);
    if (const char *env = getenv("MFGB_BATCH")) b = atoll(env);
    if (b < 1) b = 1;
    if (b > 65535) b = 65535;
    if (b > n_t) b = n_t;
    return b;
}

// exch_elems: complex64 entries of the exchange ring (max over the call's
// segments of batch * N); anc_elems: anchor records (max of batch * anchors)
static int ensure_workspace(mf_bank_s *b, int64_t exch_elems, int64_t cap, int64_t anc_elems, int64_t nblk,
                            bool capturing) {
    Workspace &w = b->ws;
    if (w.units && w.exch_elems >= exch_elems && w.n_t >= b->n && w.cap >= cap && w.anc_elems >= anc_elems &&
        w.nblk >= nblk)
        return MF_OK;
    if (capturing)
        return set_err(MF_EINVAL, "the workspace must grow: call mf_filter_bank once with these segments and "
                                  "trig_cap before capturing it");
    const int64_t ne = std::max(w.exch_elems, exch_elems), ncap = std::max(std::max(w.cap, cap), (int64_t)1);
    const int64_t na = std::max(w.anc_elems, anc_elems);
    const int64_t nbl = std::max(w.nblk, nblk);
    MF_CUDA(cudaDeviceSynchronize());
    w.release();
    MF_CUDA(dev_malloc(&w.units, sizeof(UnitInfo) * b->n));
    MF_CUDA(dev_malloc(&w.exch, sizeof(float2) * ne));
    MF_CUDA(dev_malloc(&w.anchors, sizeof(float4) * na));
    MF_CUDA(dev_malloc(&w.anchors4, sizeof(float) * na));
    MF_CUDA(dev_malloc(&w.partials, sizeof(float4) * nbl * b->n));
    MF_CUDA(dev_malloc(&w.staged, sizeof(mf_trigger) * ncap));
    MF_CUDA(dev_malloc(&w.keys, sizeof(uint64_t) * ncap));
    MF_CUDA(dev_malloc(&w.keys_tmp, sizeof(uint64_t) * ncap));
    MF_CUDA(dev_malloc(&w.idx_a, sizeof(uint32_t) * ncap));
    MF_CUDA(dev_malloc(&w.idx_b, sizeof(uint32_t) * ncap));
    MF_CUDA(dev_malloc(&w.ghist, sizeof(uint32_t) * 256 * 8));
    MF_CUDA(dev_malloc(&w.tstat, sizeof(uint64_t) * sort_tile_words(ncap)));
    MF_CUDA(dev_malloc(&w.tickets, sizeof(unsigned) * 8));
    MF_CUDA(dev_malloc(&w.counter, sizeof(unsigned long long)));
    MF_CUDA(dev_malloc(&w.status, sizeof(int)));
    MF_CUDA(cudaMemset(w.status, 0, sizeof(int)));
    MF_CUDA(dev_malloc(&w.ctl, sizeof(unsigned) * (4 + 3 * b->n)));
    w.exch_elems = ne; w.n_t = b->n; w.cap = ncap; w.anc_elems = na; w.nblk = nbl;
    return MF_OK;
}

// Persistent scheduler geometry: anchor chunks LA rounds ahead of their pass
// 1 in queue 1, anchor ring SA > LA slots, exchange ring S slots (pass 1 may
// run up to S - 1 units ahead of pass 2).  The first kSplit of the SMs start
// on queue 1 (anchors + pass 1, about 60% of the work), the rest on queue 2.
constexpr int kLA = 4, kS = 8, kSA = kLA + 4;
constexpr double kSplit = 0.60;

// Pass-1 form of a call: the bank's (autotuned) form unless MFGB_P1TILE=half
// asks for the half-width tiles of the persistent form.
static int p1_form(const mf_bank_s *b) {
    const char *e = getenv("MFGB_P1TILE");
    if (e && strcmp(e, "half") == 0) return 2;
    return b->p1_kind;
}

// Pass 2 as whole rows per warp (row length 1024 or 2048) unless MFGB_P2ROWS=0.
static bool use_rows(const mf_bank_s *b, const mf_segment_s *g, int log2N1) {
    (void)g;
    if (!pass2_rows_applies(log2N1)) return false;
    if (b->params.fft_mode != MF_FFT_FP32) return true;   // the tensor-core stage lives in the rows kernel
    if (b->p2_kind == 1) return false;
    const char *e = getenv("MFGB_P2ROWS");
    return !(e && strcmp(e, "0") == 0);
}

static bool use_persistent(const mf_bank_s *b, const mf_segment_s *g);
static bool use_fused(const mf_bank_s *b, const mf_segment_s *g);

// Column-length exponent of the split the per-batch schedule uses for this
// segment: the alternative split where the bank chose it (mf_autotune) or
// MFGB_SPLIT_ALT=1 asks for it, else the balanced one.  The persistent
// scheduler and the chi^2 paths use the balanced split.
static int filter_log2n2(const mf_bank_s *b, const mf_segment_s *g) {
    const int alt = alt_log2n2(g->log2N);
    if (alt < 0 || use_persistent(b, g) || use_fused(b, g) || b->params.fft_mode != MF_FFT_FP32) return log2_n2(g->log2N);
    const char *e = getenv("MFGB_SPLIT_ALT");
    if (e) return e[0] == '1' ? alt : log2_n2(g->log2N);
    return b->alt_split[g->log2N] ? alt : log2_n2(g->log2N);
}

static bool use_persistent(const mf_bank_s *b, const mf_segment_s *g) {
    if (g->log2N < 13 || b->params.phase_mode == MF_PHASE_FP32 || b->params.fft_mode != MF_FFT_FP32) return false;
    if (const char *e = getenv("MFGB_SCHED")) {
        if (strcmp(e, "batch") == 0 || strcmp(e, "fused") == 0) return false;
        if (strcmp(e, "persistent") == 0) return true;
    }
    return b->sched == 0;
}

// The fused scheduler (one launch of both passes through an L2-resident
// exchange ring) where it applies: N = 2^19, 2^20 on the balanced split, the
// FP64-anchor phase, FP32 FFT, a tensor map over W, the staged pass 1.
static bool use_fused(const mf_bank_s *b, const mf_segment_s *g) {
    if (b->params.phase_mode != MF_PHASE_ANCHOR || b->params.fft_mode != MF_FFT_FP32 || !g->has_tmap[0]) return false;
    if (b->n > 65535) return false;   // the anchors of every unit come from one launch (grid y)
    if (!fused_applies(g->log2N, log2_n2(g->log2N))) return false;
    if (!pass1_pf_applies(g->log2N, log2_n2(g->log2N), choose_log2D(b, g), b->params.phase_mode)) return false;
    if (const char *e = getenv("MFGB_SCHED")) return strcmp(e, "fused") == 0;
    return b->sched == 2;
}

// ring slots of the fused scheduler: 64 MiB of exchange, resident in L2
static int fused_slots(int64_t N) { return (int)std::max<int64_t>(2, ((int64_t)64 << 20) / (8 * N)); }

// Queue 1: rounds rho = -LA .. U - 1; round rho holds the anchor chunks of
// unit rho + LA and the pass-1 tiles of unit rho (those units that exist);
// consecutive rounds with the same membership form one regime.  Queue 2 holds
// the pass-2 tiles of units 0 .. U - 1 in order.  Returns false if a queue
// would not fit an int index.
static bool build_queues(int64_t U, int nA, int n1, int n2, PersistParams &P) {
    auto flags = [&](int64_t rho) {
        int f = 0;
        if (rho + kLA >= 0 && rho + kLA < U) f |= 1;
        if (rho >= 0 && rho < U) f |= 2;
        return f;
    };
    int64_t q = 0;
    int nr = 0;
    for (int64_t rho = -kLA; rho < U;) {
        const int f = flags(rho);
        int64_t end = rho + 1;
        while (end < U && flags(end) == f) ++end;
        const int64_t size = ((f & 1) ? nA : 0) + ((f & 2) ? n1 : 0);
        if (size > 0) {
            if (nr >= kMaxRegimes) return false;
            P.reg[nr].rho0 = (int)rho;
            P.reg[nr].first = (int)q;
            P.reg[nr].size = (int)size;
            P.reg[nr].rounds = (int)(end - rho);
            P.reg[nr].flags = f;
            ++nr;
            q += size * (end - rho);
            if (q >= ((int64_t)1 << 31) - 1) return false;
        }
        rho = end;
    }
    if (U * (int64_t)n2 >= ((int64_t)1 << 31) - 1) return false;
    P.n_reg = nr;
    P.n_items1 = (int)q;
    P.n_items2 = (int)(U * n2);
    P.LA = kLA;
    return true;
}

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

extern "C" int mf_filter_bank(mf_bank b, const mf_segment *segs, int n_seg, float threshold, mf_peak *peaks,
                              mf_trigger *trig, int64_t trig_cap, int64_t *n_trig, void *cuda_stream) {
    NvtxRange nvtx("mf_filter_bank");
    if (!b || !segs || n_seg < 1) return set_err(MF_EINVAL, "need a bank and n_seg >= 1 segments");
    if (!peaks || !n_trig) return set_err(MF_EINVAL, "peaks and n_trig must not be NULL");
    if (trig_cap < 0 || trig_cap > ((int64_t)1 << 31)) return set_err(MF_EINVAL, "trig_cap out of range");
    if (trig_cap > 0 && !trig) return set_err(MF_EINVAL, "trig is NULL with trig_cap > 0");
    if (!isfinite(threshold) || threshold < 0.f) return set_err(MF_EINVAL, "threshold must be finite and >= 0");
    if (n_seg > 65535) return set_err(MF_EINVAL, "at most 65535 segments per call");
    int64_t maxN = 0;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != b->device) return set_err(MF_EINVAL, "bank was created on device %d, current is %d", b->device, cur);
    for (int s = 0; s < n_seg; ++s) {
        const mf_segment_s *g = segs[s];
        if (!g) return set_err(MF_EINVAL, "segs[%d] is NULL", s);
        if (g->device != cur) return set_err(MF_EINVAL, "segs[%d] lives on device %d", s, g->device);
        if (b->params.fft_mode != MF_FFT_FP32 && g->log2N != 19 && g->log2N != 20)
            return set_err(MF_ENOTSUP, "segs[%d]: the tensor-core FFT stage needs N = 2^19 or 2^20", s);
        maxN = std::max(maxN, g->N);
        // every template's band must be non-empty: the smallest f_cut decides
        const double fc = std::min(b->fisco_min, 0.5 * g->fs);
        const int64_t lo = std::max((int64_t)1, (int64_t)ceil(b->params.f_low * (double)g->N / g->fs));
        const int64_t hi = std::min((int64_t)floor(fc * (double)g->N / g->fs) + 1, g->N / 2);
        if (hi <= lo)
            return set_err(MF_EINVAL, "segs[%d]: f_low %.3f Hz >= f_cut %.3f Hz for some template", s,
                           b->params.f_low, fc);
    }
    KeyLayout kl;
    kl.j_bits = ilog2(maxN);
    kl.seg_bits = bits_for(n_seg);
    kl.tmpl_bits = bits_for(b->n);
    const int key_bits = kl.j_bits + kl.seg_bits + kl.tmpl_bits;
    if (key_bits > 64) return set_err(MF_EINVAL, "trigger key needs %d bits", key_bits);

    // templates in flight per segment: the exchange budget over the segment's
    // length (the persistent scheduler needs its ring slots)
    std::vector<int64_t> seg_batch((size_t)n_seg);
    int64_t exch_elems = 0, anc_elems = 0, nblk = 0;
    for (int s = 0; s < n_seg; ++s) {
        int64_t bt = choose_batch(segs[s]->N, b->n, b->tuned_exch);
        if (use_persistent(b, segs[s])) bt = std::max<int64_t>(bt, std::max(kS, kSA));
        seg_batch[(size_t)s] = bt;
        const int lgD = choose_log2D(b, segs[s]);
        exch_elems = std::max(exch_elems, bt * segs[s]->N);
        anc_elems = std::max(anc_elems, 2 * bt * (((segs[s]->N / 2) >> lgD) + 2));   // two batches in flight
        if (use_fused(b, segs[s])) {   // the ring, and the anchors of every unit
            exch_elems = std::max(exch_elems, (int64_t)fused_slots(segs[s]->N) * segs[s]->N);
            anc_elems = std::max(anc_elems, b->n * anchor_slot_records(segs[s]->log2N, lgD));
        }
        const int lg2 = filter_log2n2(b, segs[s]);
        nblk = std::max(nblk, (int64_t)pass2_blocks(segs[s]->log2N, lg2));
        if ((!use_persistent(b, segs[s]) && use_rows(b, segs[s], segs[s]->log2N - lg2)) || use_fused(b, segs[s]))
            nblk = std::max(nblk, (int64_t)pass2_rows_partials(segs[s]->log2N, lg2));   // one partial per row and warp
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const bool capturing = stream_capturing(st);
    if (capturing && b->prof_on) return set_err(MF_EINVAL, "stage profiling cannot run inside a stream capture");
    int rc = ensure_workspace(b, exch_elems, trig_cap, anc_elems, nblk, capturing);
    if (rc) return rc;
    Workspace &w = b->ws;
    MF_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(unsigned long long), st));
    MF_CUDA(cudaMemsetAsync(w.status, 0, sizeof(int), st));
    const int n_t = (int)b->n;
    // descending-cost unit order (MFGB_UNIT_ORDER=bank keeps bank order); the
    // stall hook names a template, the kernels see its unit position
    const char *uo = getenv("MFGB_UNIT_ORDER");
    const int *unit_order = (uo && !strcmp(uo, "bank")) ? nullptr : b->d_order;
    const int stall_pos =
        b->stall_unit < 0 ? -1 : (unit_order ? b->pos[(size_t)b->stall_unit] : (int)b->stall_unit);
    for (int s = 0; s < n_seg; ++s) {
        const SegDev sd = seg_dev(segs[s], filter_log2n2(b, segs[s]));
        const int lgD = choose_log2D(b, segs[s]);
        const int man = (int)anchor_slot_records(segs[s]->log2N, lgD);   // records per anchor slot
        const bool rows = (!use_persistent(b, segs[s]) && use_rows(b, segs[s], sd.log2N1)) || use_fused(b, segs[s]);
        const int nbk = rows ? pass2_rows_partials(sd.log2N, sd.log2N2) : pass2_blocks(sd.log2N, sd.log2N2);
        // per-batch 1024-point FP32 rows: each row keeps only its maximum and
        // the batch's peaks are found right after its pass 2 (launch_peaks_rows)
        // (not for batches of one template, where the extra launch costs more than the search)
        const bool peaks_later = rows && !use_persistent(b, segs[s]) && !use_fused(b, segs[s]) &&
                                 seg_batch[(size_t)s] > 1 && pass2_rows_peaks_later(sd.log2N1, b->params.fft_mode);
        const bool anchors = b->params.phase_mode != MF_PHASE_FP32;
        // algorithmic bytes per template (profiling only): band of W and anchors read in pass 1
        std::vector<double> band_bytes, anc_bytes;
        if (b->prof_on) {
            band_bytes.resize((size_t)n_t);
            anc_bytes.resize((size_t)n_t);
            for (int t = 0; t < n_t; ++t) {
                const double fc = std::min(b->fisco[(size_t)t], 0.5 * sd.fs);
                int64_t lo = std::max((int64_t)1, (int64_t)ceil(b->params.f_low * (double)sd.N / sd.fs));
                int64_t hi = std::min((int64_t)floor(fc * (double)sd.N / sd.fs) + 1, sd.N / 2);
                if (hi < lo) hi = lo;
                band_bytes[(size_t)t] = 8.0 * (double)(hi - lo);
                anc_bytes[(size_t)t] = anchors ? 16.0 * (double)(((hi - 1) >> lgD) - (lo >> lgD) + 1) : 0.0;
            }
        }
        int pi = prof_begin(b, MF_STAGE_SETUP, 48.0 * n_t, st);
        MF_CUDA(launch_units(sd, b->d_tmpl, n_t, b->params.f_low, threshold, lgD, unit_order, w.units, st));
        prof_end(b, pi, st);
        count_launches(1);
        if (use_fused(b, segs[s])) {
            double by_band = 0.0, by_anc = 0.0;
            if (b->prof_on)
                for (int t = 0; t < n_t; ++t) {
                    by_band += band_bytes[(size_t)t];
                    by_anc += anc_bytes[(size_t)t];
                }
            pi = prof_begin(b, MF_STAGE_ANCHORS, by_anc, st);
            MF_CUDA(launch_anchors(sd, b->d_tmpl, w.units, 0, n_t, lgD, man, w.anchors, w.anchors4, st));
            prof_end(b, pi, st);
            MF_CUDA(cudaMemsetAsync(w.ctl, 0, sizeof(unsigned) * (4 + 2 * (size_t)n_t), st));
            double split = b->split > 0.0 ? b->split : kSplit;
            if (const char *e = getenv("MFGB_SPLIT")) split = atof(e);
            pi = prof_begin(b, MF_STAGE_FUSED, by_band + by_anc + 16.0 * (double)sd.N * n_t, st);
            MF_CUDA(launch_fused(sd, w.units, n_t, lgD, man, w.anchors, w.anchors4, w.exch, fused_slots(sd.N), split,
                                 w.ctl, w.ctl + 4, w.ctl + 4 + n_t, w.partials, s, kl, w.staged, w.keys, w.counter,
                                 std::max<int64_t>(trig_cap, 0), w.status, b->spin_limit, stall_pos, st));
            prof_end(b, pi, st);
            pi = prof_begin(b, MF_STAGE_FINAL, 16.0 * nbk * n_t, st);
            MF_CUDA(launch_reduce_peaks(sd, w.units, n_t, w.partials, nbk, s, n_seg, peaks, st));
            prof_end(b, pi, st);
            count_launches(3);
            continue;
        }
        PersistParams P;
        int n1 = 0, n2 = 0, nA = 0;
        bool persist = use_persistent(b, segs[s]);
        if (persist) {
            persist_tiles(sd.log2N, &n1, &n2);
            nA = (man + 1023) / 1024;
            persist = build_queues(n_t, nA, n1, n2, P);
        }
        if (persist) {
            // heads, abort flag, per-unit counters
            MF_CUDA(cudaMemsetAsync(w.ctl, 0, sizeof(unsigned) * (4 + 3 * (size_t)n_t), st));
            P.seg = sd;
            P.tmpl = b->d_tmpl;
            P.units = w.units;
            P.log2D = lgD;
            P.max_anc = man;
            P.nA = nA;
            P.S = kS;
            P.SA = kSA;
            P.anchors = w.anchors;
            P.anchors4 = w.anchors4;
            P.exch = w.exch;
            P.ctl = w.ctl;
            P.doneA = w.ctl + 4;
            P.done1 = w.ctl + 4 + n_t;
            P.done2 = w.ctl + 4 + 2 * (size_t)n_t;
            P.n_sm = sm_count();
            double split = b->split > 0.0 ? b->split : kSplit;
            if (const char *e = getenv("MFGB_SPLIT")) split = atof(e);
            P.split = std::min(P.n_sm - 1, std::max(1, (int)lround(split * P.n_sm)));
            P.status = w.status;
            P.partials = w.partials;
            P.staged = w.staged;
            P.keys = w.keys;
            P.counter = w.counter;
            P.cap = std::max<int64_t>(trig_cap, 0);
            P.seg_idx = s;
            P.n_seg = n_seg;
            P.kl = kl;
            P.peaks = peaks;
            P.spin_limit = b->spin_limit;
            P.stall_unit = stall_pos;
            P.stats = nullptr;
            const bool want_stats = getenv("MFGB_SCHED_STATS") != nullptr && !capturing;
            if (want_stats) {
                MF_CUDA(dev_malloc_async(&P.stats, sizeof(unsigned long long) * 12, st));
                MF_CUDA(cudaMemsetAsync(P.stats, 0, sizeof(unsigned long long) * 12, st));
            }
            double by = 16.0 * (double)sd.N * n_t;
            if (b->prof_on)
                for (int t = 0; t < n_t; ++t) by += band_bytes[(size_t)t] + anc_bytes[(size_t)t];
            const int grid = std::max(1, persist_blocks_per_sm(sd.log2N)) * sm_count();
            pi = prof_begin(b, MF_STAGE_FUSED, by, st);
            MF_CUDA(launch_persistent(P, grid, st));
            prof_end(b, pi, st);
            count_launches(1);
            if (want_stats) {   // diagnostics only: synchronises
                unsigned long long h[12];
                MF_CUDA(cudaMemcpyAsync(h, P.stats, sizeof(h), cudaMemcpyDeviceToHost, st));
                MF_CUDA(cudaStreamSynchronize(st));
                cudaFreeAsync(P.stats, st);
                const char *nm[3] = {"anchors", "pass1", "pass2"};
                for (int ph = 0; ph < 3; ++ph)
                    fprintf(stderr, "mfgb sched %-7s items %8llu waited %8llu  wait %.3e cyc\n", nm[ph],
                            h[4 * ph + 2], h[4 * ph + 3], (double)h[4 * ph + 1]);
            }
            pi = prof_begin(b, MF_STAGE_FINAL, 16.0 * nbk * n_t, st);
            MF_CUDA(launch_reduce_peaks(sd, w.units, n_t, w.partials, nbk, s, n_seg, peaks, st));
            prof_end(b, pi, st);
            count_launches(1);
            continue;
        }
        const int64_t batch = seg_batch[(size_t)s];
        // Anchors of batch i + 1 run on a side stream beside pass 2 of batch i,
        // into the other of two anchor slots (its previous reader, pass 1 of
        // batch i - 1, finished before pass 1 of batch i, which the side
        // stream waits for).  Stage profiling keeps everything on one stream.
        const bool overlap = anchors && !b->prof_on && batch < n_t;
        if (overlap && !b->side) {
            if (capturing) return set_err(MF_EINVAL, "call mf_filter_bank once before capturing it");
            MF_CUDA(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
            MF_CUDA(cudaEventCreateWithFlags(&b->ev_p1, cudaEventDisableTiming));
            MF_CUDA(cudaEventCreateWithFlags(&b->ev_anc, cudaEventDisableTiming));
        }
        const int64_t slot_elems = batch * man;
        for (int u0 = 0, bi = 0; u0 < n_t; u0 += (int)batch, ++bi) {
            const int nb = (int)std::min<int64_t>(batch, n_t - u0);
            const int64_t aoff = overlap ? (bi & 1) * slot_elems : 0;
            double by_band = 0.0, by_anc = 0.0;
            if (b->prof_on)
                for (int u = u0; u < u0 + nb; ++u) {
                    const size_t t = unit_order ? (size_t)b->order[(size_t)u] : (size_t)u;
                    by_band += band_bytes[t];
                    by_anc += anc_bytes[t];
                }
            const double exch_bytes = 8.0 * (double)sd.N * nb;
            if (anchors && (!overlap || bi == 0)) {
                pi = prof_begin(b, MF_STAGE_ANCHORS, by_anc, st);
                MF_CUDA(launch_anchors(sd, b->d_tmpl, w.units, u0, nb, lgD, man, w.anchors + aoff, w.anchors4 + aoff,
                                       st));
                prof_end(b, pi, st);
                count_launches(1);
            } else if (overlap) {
                MF_CUDA(cudaStreamWaitEvent(st, b->ev_anc, 0));
            }
            pi = prof_begin(b, MF_STAGE_PASS1, by_band + by_anc + exch_bytes, st);
            MF_CUDA(launch_pass1(sd, w.units, u0, nb, lgD, man, w.anchors + aoff, w.anchors4 + aoff, w.exch,
                                 b->params.phase_mode, b->d_tmpl, p1_form(b), w.status, b->spin_limit, st));
            prof_end(b, pi, st);
            if (overlap && u0 + batch < n_t) {
                const int u1 = u0 + (int)batch;
                const int nb1 = (int)std::min<int64_t>(batch, n_t - u1);
                const int64_t aoff1 = ((bi + 1) & 1) * slot_elems;
                MF_CUDA(cudaEventRecord(b->ev_p1, st));
                MF_CUDA(cudaStreamWaitEvent(b->side, b->ev_p1, 0));
                MF_CUDA(launch_anchors(sd, b->d_tmpl, w.units, u1, nb1, lgD, man, w.anchors + aoff1,
                                       w.anchors4 + aoff1, b->side));
                MF_CUDA(cudaEventRecord(b->ev_anc, b->side));
                count_launches(1);
            }
            pi = prof_begin(b, MF_STAGE_PASS2, exch_bytes, st);
            if (rows)
                MF_CUDA(launch_pass2_rows(sd, w.units, u0, nb, w.exch, w.partials, s, kl, w.staged, w.keys, w.counter,
                                          std::max<int64_t>(trig_cap, 0), w.status, b->spin_limit, sm_count(),
                                          b->params.fft_mode, stall_pos, peaks_later, st));
            else
                MF_CUDA(launch_pass2(sd, w.units, u0, nb, w.exch, w.partials, s, kl, w.staged, w.keys, w.counter,
                                     std::max<int64_t>(trig_cap, 0), st));
            prof_end(b, pi, st);
            count_launches(2);
            if (peaks_later) {   // the batch's peaks, while its exchange is still there
                pi = prof_begin(b, MF_STAGE_FINAL, 16.0 * nbk * nb, st);
                MF_CUDA(launch_peaks_rows(sd, w.units, u0, nb, n_t, w.exch, w.partials, s, n_seg, peaks, st));
                prof_end(b, pi, st);
                count_launches(1);
            }
        }
        if (!peaks_later) {
            pi = prof_begin(b, MF_STAGE_FINAL, 16.0 * nbk * n_t, st);
            MF_CUDA(launch_reduce_peaks(sd, w.units, n_t, w.partials, nbk, s, n_seg, peaks, st));
            prof_end(b, pi, st);
            count_launches(1);
        }
    }
    int pf = prof_begin(b, MF_STAGE_FINAL, 0.0, st);
    MF_CUDA(launch_sort_triggers(w.counter, std::max<int64_t>(trig_cap, 0), key_bits, w.staged, w.keys,
                                 w.keys_tmp, w.idx_a, w.idx_b, w.ghist, w.tstat, w.tickets, trig, nullptr, n_trig,
                                 w.status, sm_count(), b->spin_limit, st));
    prof_end(b, pf, st);
    count_launches(sort_launches(key_bits));
    return MF_OK;
}

extern "C" int mf_fft_c2c(const void *x, void *y, int64_t N, int64_t batch, int sign, void *cuda_stream) {
    if (!x || !y) return set_err(MF_EINVAL, "NULL argument");
    if (!is_pow2_in(N, 10, 22)) return set_err(MF_EINVAL, "N = %lld must be a power of two in [2^10, 2^22]", (long long)N);
    if (batch < 1) return set_err(MF_EINVAL, "batch < 1");
    if (sign != 1 && sign != -1) return set_err(MF_EINVAL, "sign must be +1 or -1");
    if (((uintptr_t)x | (uintptr_t)y) & 7) return set_err(MF_EINVAL, "x and y must be 8-byte aligned complex64 arrays");
    int r0 = ensure_device_init();
    if (r0) return r0;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (fft_c2c_single_pass(N)) {   // whole sequences per CTA: no exchange
        MF_CUDA(launch_fft_c2c_single((const float2 *)x, (float2 *)y, N, batch, sign, st));
        count_launches(1);
        return MF_OK;
    }
    if (stream_capturing(st)) return set_err(MF_EINVAL, "mf_fft_c2c allocates its exchange and cannot be captured");
    const int64_t chunk = std::min<int64_t>({batch, std::max<int64_t>(1, kScratchBudget / (8 * N)), 65535});
    float2 *exch = nullptr;
    cudaError_t e = dev_malloc_async(&exch, sizeof(float2) * N * chunk, st);
    int launches = 0;
    for (int64_t b0 = 0; b0 < batch && e == cudaSuccess; b0 += chunk) {
        const int nb = (int)std::min<int64_t>(chunk, batch - b0);
        e = launch_fft_c2c((const float2 *)x + b0 * N, (float2 *)y + b0 * N, N, nb, sign, exch, st);
        launches += 2;
    }
    if (exch) cudaFreeAsync(exch, st);
    if (e != cudaSuccess)
        return set_err(e == cudaErrorMemoryAllocation ? MF_ENOMEM : MF_ECUDA, "fft_c2c: %s", cudaGetErrorString(e));
    count_launches(launches);
    return MF_OK;
}

extern "C" int mf_chisq_series(mf_bank b, mf_segment seg, const int32_t *tmpl, int64_t n, int p, float *chisq,
                               int64_t *edges, void *cuda_stream) {
    NvtxRange nvtx("mf_chisq_series");
    if (!b || !seg || !tmpl || !chisq) return set_err(MF_EINVAL, "NULL argument");
    if (n < 1 || n > ((int64_t)1 << 24)) return set_err(MF_EINVAL, "n = %lld outside [1, 2^24]", (long long)n);
    if (p < 1 || p > kChisqMaxBands) return set_err(MF_EINVAL, "p = %d outside [1, %d]", p, kChisqMaxBands);
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != b->device || seg->device != cur) return set_err(MF_EINVAL, "bank and segment must live on the current device");
    {
        const double fc = std::min(b->fisco_min, 0.5 * seg->fs);
        const int64_t lo = std::max((int64_t)1, (int64_t)ceil(b->params.f_low * (double)seg->N / seg->fs));
        const int64_t hi = std::min((int64_t)floor(fc * (double)seg->N / seg->fs) + 1, seg->N / 2);
        if (hi <= lo) return set_err(MF_EINVAL, "f_low >= f_cut for some template of the bank");
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (stream_capturing(st)) return set_err(MF_EINVAL, "mf_chisq_series allocates scratch and cannot be captured");
    const SegDev sd = seg_dev(seg);
    const int lgD = choose_log2D(b, seg);
    const int man = (int)anchor_slot_records(seg->log2N, lgD);   // records per anchor slot
    const int n_t = (int)b->n;
    // 1024-point rows: every sub-band's exchange of a batch first, then one
    // rows kernel over all of them (p + 1 exchanges per template in flight)
    const bool rows = chisq_rows_applies(seg->log2N);
    const int64_t budget = b->tuned_exch > 0 ? b->tuned_exch : kExchBudget;
    const int64_t batch = rows ? std::max<int64_t>(1, std::min<int64_t>(n, budget / (8 * seg->N * (p + 1))))
                               : std::min<int64_t>(n, choose_batch(seg->N, n, budget));
    const bool anchors = b->params.phase_mode != MF_PHASE_FP32;
    if (rows && !b->chi_status) MF_CUDA(dev_malloc(&b->chi_status, sizeof(int)));
    if (b->chi_status) MF_CUDA(cudaMemsetAsync(b->chi_status, 0, sizeof(int), st));
    // With the persistent pass 1, one launch per batch covers all p + 1 bands:
    // unit slot l nb + s is band l of template u0 + s (a band-major copy of the
    // batch's units), reading the copy of its template's anchors that the
    // anchor launch stores for each band.
    const bool merged = rows && p1_form(b) != 1 && pass1_pf_applies(sd.log2N, sd.log2N2, lgD, b->params.phase_mode);
    UnitInfo *all = nullptr, *units = nullptr, *mu = nullptr;
    float4 *anc = nullptr;
    float *anc4 = nullptr;
    float2 *exch = nullptr;
    cudaError_t e = dev_malloc_async(&all, sizeof(UnitInfo) * n_t, st);
    if (e == cudaSuccess) e = dev_malloc_async(&units, sizeof(UnitInfo) * (size_t)(p + 1) * n, st);
    if (e == cudaSuccess && merged) e = dev_malloc_async(&mu, sizeof(UnitInfo) * (size_t)(p + 1) * batch, st);
    const int64_t anc_slots = batch * (merged ? p + 1 : 1);
    if (e == cudaSuccess) e = dev_malloc_async(&anc, sizeof(float4) * man * anc_slots, st);
    if (e == cudaSuccess) e = dev_malloc_async(&anc4, sizeof(float) * man * anc_slots, st);
    if (e == cudaSuccess) e = dev_malloc_async(&exch, sizeof(float2) * seg->N * batch * (rows ? p + 1 : 1), st);
    int launches = 0;
    if (e == cudaSuccess) e = launch_units(sd, b->d_tmpl, n_t, b->params.f_low, 0.f, lgD, nullptr, all, st);
    if (e == cudaSuccess) e = launch_chisq_units(sd, all, n_t, tmpl, (int)n, p, units, edges, st);
    launches += 2;
    const UnitInfo *full = units + (size_t)p * n;
    for (int64_t u0 = 0; u0 < n && e == cudaSuccess; u0 += batch) {
        const int nb = (int)std::min<int64_t>(batch, n - u0);
        if (anchors) {
            e = launch_anchors(sd, b->d_tmpl, full, (int)u0, nb, lgD, man, anc, anc4, st, merged ? p + 1 : 1);
            ++launches;
        }
        if (rows) {
            if (merged) {
                if (e == cudaSuccess)
                    e = cudaMemcpy2DAsync(mu, sizeof(UnitInfo) * nb, units + u0, sizeof(UnitInfo) * n,
                                          sizeof(UnitInfo) * nb, p + 1, cudaMemcpyDeviceToDevice, st);
                if (e == cudaSuccess)
                    e = launch_pass1(sd, mu, 0, (p + 1) * nb, lgD, man, anc, anc4, exch, b->params.phase_mode,
                                     b->d_tmpl, p1_form(b), b->chi_status, b->spin_limit, st, true);
                ++launches;
            }
            for (int l = 0; !merged && l <= p && e == cudaSuccess; ++l) {
                e = launch_pass1(sd, units + (size_t)l * n, (int)u0, nb, lgD, man, anc, anc4,
                                 exch + (size_t)l * nb * seg->N, b->params.phase_mode, b->d_tmpl, p1_form(b),
                                 b->chi_status, b->spin_limit, st);
                ++launches;
            }
            if (e == cudaSuccess)
                e = launch_chisq_rows(sd, exch, full, (int)u0, nb, p, chisq, b->chi_status, b->spin_limit,
                                      (int)b->stall_unit, sm_count(), st);
            ++launches;
            continue;
        }
        for (int l = 0; l <= p && e == cudaSuccess; ++l) {
            const UnitInfo *ul = units + (size_t)l * n;
            e = launch_pass1(sd, ul, (int)u0, nb, lgD, man, anc, anc4, exch, b->params.phase_mode, b->d_tmpl,
                             p1_form(b), b->chi_status, b->spin_limit, st);
            if (e == cudaSuccess)
                e = launch_chisq_pass2(sd, ul, (int)u0, nb, exch, chisq, l == p ? 2 : (l == 0 ? 0 : 1), p, st);
            launches += 2;
        }
    }
    if (all) cudaFreeAsync(all, st);
    if (units) cudaFreeAsync(units, st);
    if (mu) cudaFreeAsync(mu, st);
    if (anc) cudaFreeAsync(anc, st);
    if (anc4) cudaFreeAsync(anc4, st);
    if (exch) cudaFreeAsync(exch, st);
    if (e != cudaSuccess)
        return set_err(e == cudaErrorMemoryAllocation ? MF_ENOMEM : MF_ECUDA, "chisq_series: %s", cudaGetErrorString(e));
    count_launches(launches);
    return MF_OK;
}

extern "C" int mf_cluster_triggers(const mf_trigger *trig, const int64_t *n_trig, int64_t trig_cap, int64_t n_tmpl,
                                   int n_seg, int64_t max_N, int32_t window, mf_event *events, int64_t ev_cap,
                                   int64_t *n_events, void *cuda_stream) {
    if (!trig || !n_trig || !n_events || (ev_cap > 0 && !events)) return set_err(MF_EINVAL, "NULL argument");
    if (trig_cap < 1 || trig_cap > ((int64_t)1 << 31)) return set_err(MF_EINVAL, "trig_cap out of range");
    if (ev_cap < 0 || window < 0 || n_tmpl < 1 || n_seg < 1 || max_N < 2)
        return set_err(MF_EINVAL, "ev_cap, window, n_tmpl, n_seg or max_N out of range");
    KeyLayout kl;
    kl.j_bits = ilog2(max_N) + ((max_N & (max_N - 1)) ? 1 : 0);
    kl.seg_bits = bits_for(n_seg);
    kl.tmpl_bits = bits_for(n_tmpl);
    const int key_bits = kl.j_bits + kl.seg_bits + kl.tmpl_bits;
    if (key_bits > 64) return set_err(MF_EINVAL, "cluster key needs %d bits", key_bits);
    int r0 = ensure_device_init();
    if (r0) return r0;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int64_t cap = trig_cap;
    const int64_t nb = cluster_scan_blocks(cap);
    ClusterScratch w;
    std::vector<void *> bufs;
    cudaError_t e = cudaSuccess;
    auto get = [&](auto **ptr, size_t bytes) {
        void *q = nullptr;
        if (e == cudaSuccess) e = dev_malloc_async(&q, bytes, st);
        if (e == cudaSuccess) bufs.push_back(q);
        *ptr = (std::remove_pointer_t<decltype(ptr)>)q;
    };
    get(&w.flag, sizeof(uint32_t) * cap);
    get(&w.incl, sizeof(uint32_t) * cap);
    get(&w.bsum, sizeof(uint32_t) * nb);
    get(&w.members, sizeof(uint32_t) * cap);
    get(&w.wsum, sizeof(uint32_t) * cap);
    get(&w.rep_count, sizeof(uint32_t) * cap);
    get(&w.idx_a, sizeof(uint32_t) * cap);
    get(&w.idx_b, sizeof(uint32_t) * cap);
    get(&w.perm, sizeof(uint32_t) * cap);
    get(&w.ghist, sizeof(uint32_t) * 256 * 8);
    get(&w.best, sizeof(unsigned long long) * cap);
    get(&w.rep, sizeof(mf_trigger) * cap);
    get(&w.sorted, sizeof(mf_trigger) * cap);
    get(&w.keys, sizeof(uint64_t) * cap);
    get(&w.keys_tmp, sizeof(uint64_t) * cap);
    get(&w.tstat, sizeof(uint64_t) * sort_tile_words(cap));
    get(&w.tickets, sizeof(unsigned) * 8);
    get(&w.n_c, sizeof(int64_t));
    get(&w.n_sorted, sizeof(int64_t));
    get(&w.status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(w.status, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = launch_cluster(trig, n_trig, cap, window, kl, w, events, ev_cap, n_events, sm_count(), 4000000, st);
    for (void *q : bufs) cudaFreeAsync(q, st);
    if (e != cudaSuccess)
        return set_err(e == cudaErrorMemoryAllocation ? MF_ENOMEM : MF_ECUDA, "cluster_triggers: %s",
                       cudaGetErrorString(e));
    count_launches(cluster_launches(key_bits));
    return MF_OK;
}

extern "C" int mf_chisq_points(mf_bank b, const mf_segment *segs, int n_seg, const int32_t *rows, int64_t stride,
                               int64_t n, int p, float *chisq, void *cuda_stream) {
    if (!b || !segs || !rows || !chisq) return set_err(MF_EINVAL, "NULL argument");
    if (n < 0 || stride < 3) return set_err(MF_EINVAL, "n < 0 or stride < 3");
    if (p < 1 || p > kChisqMaxBands) return set_err(MF_EINVAL, "p = %d outside [1, %d]", p, kChisqMaxBands);
    if (n_seg < 1 || n_seg > kRefineMaxSegs) return set_err(MF_EINVAL, "n_seg outside [1, %d]", kRefineMaxSegs);
    if (n == 0) return MF_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    if (b->device != cur) return set_err(MF_EINVAL, "bank lives on device %d", b->device);
    std::vector<SegDev> sd((size_t)n_seg);
    for (int s = 0; s < n_seg; ++s) {
        if (!segs[s] || segs[s]->device != cur) return set_err(MF_EINVAL, "segs[%d] is NULL or on another device", s);
        sd[(size_t)s] = seg_dev(segs[s]);
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int64_t chunk = std::min<int64_t>(n, 65535);
    const int bpr = (int)std::max<int64_t>(4, std::min<int64_t>(64, (4 * (int64_t)sm_count() + chunk - 1) / chunk));
    double2 *partial = nullptr;
    cudaError_t e = dev_malloc_async(&partial, sizeof(double2) * (size_t)bpr * chunk * p, st);
    int launches = 0;
    for (int64_t i0 = 0; i0 < n && e == cudaSuccess; i0 += chunk) {
        const int64_t m = std::min<int64_t>(chunk, n - i0);
        e = launch_chisq_points(sd.data(), n_seg, b->d_tmpl, (int)b->n, b->params.f_low, b->params.phase_mode,
                                rows + i0 * stride, stride, m, p, bpr, partial, chisq + i0, st);
        launches += 2;
    }
    if (partial) cudaFreeAsync(partial, st);
    if (e != cudaSuccess)
        return set_err(e == cudaErrorMemoryAllocation ? MF_ENOMEM : MF_ECUDA, "chisq_points: %s", cudaGetErrorString(e));
    count_launches(launches);
    return MF_OK;
}

extern "C" int mf_debug_status(uint32_t *word, int *enabled) {
    if (!word) return set_err(MF_EINVAL, "NULL argument");
#ifdef MFGB_DEBUG
    if (enabled) *enabled = 1;
#else
    if (enabled) *enabled = 0;
#endif
    int r0 = ensure_device_init();
    if (r0) return r0;
    MF_CUDA(cudaDeviceSynchronize());
    unsigned all = 0, w = 0;
    cudaError_t (*readers[])(unsigned *) = {dbg_read_filter, dbg_read_pass1, dbg_read_rows,
                                            dbg_read_persist, dbg_read_chisq, dbg_read_prep, dbg_read_fused};
    for (auto rd : readers) {
        MF_CUDA(rd(&w));
        all |= w;
    }
    *word = all;
    return MF_OK;
}

extern "C" int mf_bank_debug_stall(mf_bank b, int64_t unit, int64_t spin_limit) {
    if (!b) return set_err(MF_EINVAL, "NULL bank");
    if (unit >= b->n) return set_err(MF_EINVAL, "unit out of range");
    b->stall_unit = unit < 0 ? -1 : unit;
    b->spin_limit = spin_limit > 0 ? spin_limit : 4000000;
    return MF_OK;
}

extern "C" int mf_bank_profile(mf_bank b, int on) {
    if (!b) return set_err(MF_EINVAL, "NULL bank");
    b->prof_on = on != 0;
    return MF_OK;
}

extern "C" int mf_bank_profile_read(mf_bank b, double *ms, double *bytes, int64_t *launches) {
    if (!b || !ms || !bytes || !launches) return set_err(MF_EINVAL, "NULL argument");
    for (int i = 0; i < MF_N_STAGES; ++i) { ms[i] = 0.0; bytes[i] = 0.0; launches[i] = 0; }
    for (auto &r : b->prof) {
        MF_CUDA(cudaEventSynchronize(r.b));
        float t = 0.f;
        MF_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
        ms[r.stage] += t;
        bytes[r.stage] += r.bytes;
        launches[r.stage] += 1;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    b->prof.clear();
    return MF_OK;
}

extern "C" int mf_bank_check(mf_bank b, void *cuda_stream) {
    if (!b) return set_err(MF_EINVAL, "NULL bank");
    MF_CUDA(cudaStreamSynchronize((cudaStream_t)cuda_stream));
    if (b->chi_status) {
        int cs = 0;
        MF_CUDA(cudaMemcpy(&cs, b->chi_status, sizeof(int), cudaMemcpyDeviceToHost));
        if (cs & 2) return set_err(MF_ETIMEOUT, "a bounded device wait expired in the last mf_chisq_series");
    }
    if (!b->ws.status) return MF_OK;
    int st = 0;
    MF_CUDA(cudaMemcpy(&st, b->ws.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & 2) return set_err(MF_ETIMEOUT, "a bounded device wait expired in the last mf_filter_bank");
    if (st & 1) return set_err(MF_EOVERFLOW, "more triggers than trig_cap in the last mf_filter_bank");
    return MF_OK;
}

// ---------------------------------------------------------------------------
// autotuner: time candidate schedules of mf_filter_bank on this bank and these
// segments and keep the fastest
// ---------------------------------------------------------------------------
extern "C" int mf_autotune(mf_bank b, const mf_segment *segs, int n_seg, float threshold, int repeats,
                           const char *cache_path, void *cuda_stream) {
    NvtxRange nvtx("mf_autotune");
    if (!b || !segs || n_seg < 1) return set_err(MF_EINVAL, "need a bank and n_seg >= 1 segments");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (repeats < 1) repeats = 2;
    struct Cand { int sched; int64_t exch; double split; int p1, p2; };
    std::vector<Cand> cands;
    if (b->params.fft_mode == MF_FFT_FP32)   // the tensor-core stage runs in the per-batch rows kernel only
        for (double sp : {0.55, 0.60, 0.65}) cands.push_back({0, 0, sp, 0, 0});
    int64_t maxN = 0;
    for (int s = 0; s < n_seg; ++s) maxN = std::max(maxN, segs[s]->N);
    // per-batch launches: exchange budget x the kernel forms of the two passes
    // (the per-tile forms only where the other form would apply to some segment)
    bool any_pf = false, any_rows = false;
    for (int s = 0; s < n_seg; ++s) {
        const int lgD = choose_log2D(b, segs[s]);
        const int lg2 = log2_n2(segs[s]->log2N);
        any_pf = any_pf || pass1_pf_applies(segs[s]->log2N, lg2, lgD, b->params.phase_mode);
        any_rows = any_rows || (pass2_rows_applies(segs[s]->log2N - lg2) && b->params.fft_mode == MF_FFT_FP32);
    }
    // the fused scheduler, where it applies to some segment of the call
    bool any_fused = false;
    for (int s = 0; s < n_seg; ++s) {
        const int saved = b->sched;
        b->sched = 2;
        any_fused = any_fused || use_fused(b, segs[s]);
        b->sched = saved;
    }
    if (any_fused)
        for (double sp : {0.58, 0.60, 0.62}) cands.push_back({2, 0, sp, 0, 0});
    for (int64_t mib : {512, 1024, 2048, 4096, 8192}) {
        cands.push_back({1, mib << 20, 0.60, 0, 0});
        if (any_pf) cands.push_back({1, mib << 20, 0.60, 1, 0});
        if (any_pf) cands.push_back({1, mib << 20, 0.60, 2, 0});
        if (any_rows) cands.push_back({1, mib << 20, 0.60, 0, 1});
    }
    const int64_t cap = 1 << 16;
    mf_peak *pk = nullptr;
    mf_trigger *tr = nullptr;
    int64_t *nt = nullptr;
    {
        cudaError_t ea = dev_malloc(&pk, sizeof(mf_peak) * b->n * n_seg);
        if (ea == cudaSuccess) ea = dev_malloc(&tr, sizeof(mf_trigger) * cap);
        if (ea == cudaSuccess) ea = dev_malloc(&nt, sizeof(int64_t));
        if (ea != cudaSuccess) {
            cudaFree(pk);
            cudaFree(tr);
            cudaFree(nt);
            return set_err(ea == cudaErrorMemoryAllocation ? MF_ENOMEM : MF_ECUDA, "autotune: %s",
                           cudaGetErrorString(ea));
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // time one configuration of the bank on these segments: 1 + repeats calls, ms per call
    auto time_calls = [&](const mf_segment *sg, int ns, float &ms) -> int {
        int r = mf_filter_bank(b, sg, ns, threshold, pk, tr, cap, nt, cuda_stream);   // warm-up, sizes workspace
        if (r) return r;
        cudaEventRecord(e0, st);
        for (int k = 0; k < repeats && !r; ++k) r = mf_filter_bank(b, sg, ns, threshold, pk, tr, cap, nt, cuda_stream);
        cudaEventRecord(e1, st);
        if (r) return r;
        if (cudaEventSynchronize(e1) != cudaSuccess) return set_err(MF_ECUDA, "autotune timing");
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)repeats;
        return MF_OK;
    };
    // 1. the four-step split per segment length, on the per-batch schedule with
    // the default kernel forms: balanced N1 x N2 or the alternative split
    const int saved_sched0 = b->sched, saved_p1 = b->p1_kind, saved_p2 = b->p2_kind;
    b->sched = 1;
    b->p1_kind = 0;
    b->p2_kind = 0;
    std::vector<int> lengths;
    int rc0 = MF_OK;
    for (int s = 0; s < n_seg && !rc0; ++s) {
        const int lg = segs[s]->log2N;
        if (alt_log2n2(lg) < 0 || std::find(lengths.begin(), lengths.end(), lg) != lengths.end()) continue;
        if (b->params.fft_mode != MF_FFT_FP32) continue;
        lengths.push_back(lg);
        std::vector<mf_segment> sub;
        for (int q = 0; q < n_seg; ++q)
            if (segs[q]->log2N == lg) sub.push_back(segs[q]);
        float ms_bal = 0.f, ms_alt = 0.f;
        b->alt_split[lg] = 0;
        rc0 = time_calls(sub.data(), (int)sub.size(), ms_bal);
        if (rc0) break;
        b->alt_split[lg] = 1;
        rc0 = time_calls(sub.data(), (int)sub.size(), ms_alt);
        b->alt_split[lg] = (rc0 == MF_OK && ms_alt < ms_bal) ? 1 : 0;
    }
    b->sched = saved_sched0;
    b->p1_kind = saved_p1;
    b->p2_kind = saved_p2;
    if (rc0) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(pk);
        cudaFree(tr);
        cudaFree(nt);
        return rc0;
    }
    const int saved_sched = b->sched;
    const int64_t saved_exch = b->tuned_exch;
    const double saved_split = b->split;
    float best_ms = 1e30f;
    Cand best = {saved_sched, saved_exch, saved_split, b->p1_kind, b->p2_kind};
    int rc = MF_OK;
    for (const Cand &c : cands) {
        b->sched = c.sched;
        b->tuned_exch = c.exch;
        b->split = c.split;
        b->p1_kind = c.p1;
        b->p2_kind = c.p2;
        float ms = 0.f;
        rc = time_calls(segs, n_seg, ms);
        if (rc) break;
        if (ms < best_ms) { best_ms = ms; best = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(pk);
    cudaFree(tr);
    cudaFree(nt);
    b->sched = best.sched;
    b->tuned_exch = best.exch;
    b->split = best.split;
    b->p1_kind = best.p1;
    b->p2_kind = best.p2;
    if (rc) return rc;
    if (cache_path && cache_path[0]) {
        FILE *f = fopen(cache_path, "w");
        if (!f) return set_err(MF_EINVAL, "cannot write %s", cache_path);
        const int64_t ex = best.exch > 0 ? best.exch : kExchBudget;
        std::string sp = "{";
        std::vector<std::pair<int, int>> all_lg;   // (log2 N, the column length the tuned bank uses)
        for (int s = 0; s < n_seg; ++s) {
            const int lg = segs[s]->log2N;
            bool seen = false;
            for (const auto &q : all_lg) seen = seen || q.first == lg;
            if (!seen) all_lg.push_back({lg, filter_log2n2(b, segs[s])});
        }
        std::sort(all_lg.begin(), all_lg.end());
        for (size_t i = 0; i < all_lg.size(); ++i) {
            const int lg = all_lg[i].first;
            const int l2 = all_lg[i].second;
            char buf[96];
            snprintf(buf, sizeof(buf), "%s\"%lld\": \"%lld x %lld\"", i ? ", " : "", (long long)1 << lg,
                     (long long)1 << (lg - l2), (long long)1 << l2);
            sp += buf;
        }
        sp += "}";
        fprintf(f, "{\"N\": %lld, \"templates\": %lld, \"segments\": %d, \"scheduler\": \"%s\", "
                   "\"exchange_mib\": %lld, \"batch_at_max_N\": %lld, \"split\": %.3f, \"pass1\": \"%s\", "
                   "\"pass2\": \"%s\", \"n1_x_n2\": %s, \"candidates\": %d, \"ms_per_call\": %.4f}\n",
                (long long)maxN, (long long)b->n, n_seg,
                best.sched == 0 ? "persistent" : (best.sched == 2 ? "fused" : "batch"),
                (long long)(ex >> 20), (long long)choose_batch(maxN, b->n, ex), best.split,
                best.sched != 1 ? "fused"
                                : (best.p1 == 0 ? "persistent-staged" : (best.p1 == 2 ? "persistent-staged-half-tile"
                                                                                        : "per-tile")),
                best.sched != 1 ? "fused" : (best.p2 == 0 ? "rows" : "per-tile"), sp.c_str(),
                (int)(cands.size() + 2 * lengths.size()), best_ms);
        fclose(f);
    }
    return MF_OK;
}

// ---------------------------------------------------------------------------
// synthesis
// ---------------------------------------------------------------------------
extern "C" int mf_synth_segment(const double *g, int64_t N, double fs, double f_low, const double *psd,
                                double psd_f0, double psd_S0, const mf_injection *inj, int64_t n_inj,
                                double noise_scale, float *s_out, void *cuda_stream) {
    if (!g || !s_out) return set_err(MF_EINVAL, "g and s_out must not be NULL");
    if (!is_pow2_in(N, 10, 22)) return set_err(MF_EINVAL, "N must be a power of two in [2^10, 2^22]");
    if (!(fs > 0.0) || !(f_low > 0.0) || !isfinite(noise_scale)) return set_err(MF_EINVAL, "bad fs/f_low/noise_scale");
    if (n_inj < 0 || (n_inj > 0 && !inj) || n_inj > 4096) return set_err(MF_EINVAL, "bad injections");
    if (!psd && (!(psd_f0 > 0.0) || !(psd_S0 > 0.0))) return set_err(MF_EINVAL, "psd_f0 and psd_S0 must be > 0");
    int r0 = ensure_device_init();
    if (r0) return r0;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int64_t half = N / 2;
    std::vector<double> rec((size_t)std::max<int64_t>(n_inj, 1) * 10, 0.0);
    for (int64_t i = 0; i < n_inj; ++i) {
        const mf_injection &J = inj[i];
        if (!(J.m1 > 0.0) || !(J.m2 > 0.0) || !isfinite(J.snr) || !isfinite(J.phi))
            return set_err(MF_EINVAL, "injection %lld: bad parameters", (long long)i);
        double t[kTmplStride];
        template_constants(J.m1, J.m2, t);
        double *r = &rec[(size_t)i * 10];
        r[0] = t[TF_C1]; r[1] = t[TF_C2]; r[2] = t[TF_C3]; r[3] = t[TF_C5];
        const double fc = std::min(t[TF_FISCO], 0.5 * fs);
        int64_t lo = (int64_t)ceil(f_low * (double)N / fs), hi = (int64_t)floor(fc * (double)N / fs) + 1;
        if (lo < 1) lo = 1;
        if (hi > half) hi = half;
        if (hi <= lo) return set_err(MF_EINVAL, "injection %lld: empty band", (long long)i);
        r[4] = (double)lo; r[5] = (double)hi;
        int64_t j0 = J.j0 % N;
        if (j0 < 0) j0 += N;
        r[6] = (double)j0;
        r[7] = J.phi / (2.0 * M_PI);
        r[8] = J.snr;
    }
    double *inj_dev = nullptr, *q = nullptr, *P = nullptr, *btmp = nullptr, *psd_dev = nullptr;
    float2 *Y = nullptr, *exch = nullptr;
    const int64_t nbt = prefix_block_tmp_count(half);
    cudaError_t e = dev_malloc_async(&inj_dev, sizeof(double) * rec.size(), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(inj_dev, rec.data(), sizeof(double) * rec.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = dev_malloc_async(&q, sizeof(double) * half, st);
    if (e == cudaSuccess) e = dev_malloc_async(&P, sizeof(double) * (half + 1), st);
    if (e == cudaSuccess) e = dev_malloc_async(&btmp, sizeof(double) * nbt, st);
    if (e == cudaSuccess) e = dev_malloc_async(&Y, sizeof(float2) * half, st);
    if (e == cudaSuccess) e = dev_malloc_async(&exch, sizeof(float2) * N, st);
    if (e == cudaSuccess && psd) {
        e = dev_malloc_async(&psd_dev, sizeof(double) * (half + 1), st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(psd_dev, psd, sizeof(double) * (half + 1), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = launch_psd_weights(nullptr, psd_dev, psd_f0, psd_S0, N, fs, q, st);
    if (e == cudaSuccess) e = launch_prefix_f64(q, half, P, btmp, st);
    if (e == cudaSuccess)
        e = launch_synth_spectrum(g, N, fs, f_low, psd_dev, psd_f0, psd_S0, inj_dev, n_inj, P, noise_scale, Y, st);
    if (e == cudaSuccess) e = launch_inverse_real_fft(Y, N, 2.0 * fs / (double)N, exch, s_out, st);
    if (e == cudaSuccess) count_launches(7);   // weights, 3 scan kernels, spectrum, 2 FFT passes
    if (inj_dev) cudaFreeAsync(inj_dev, st);
    if (q) cudaFreeAsync(q, st);
    if (P) cudaFreeAsync(P, st);
    if (btmp) cudaFreeAsync(btmp, st);
    if (Y) cudaFreeAsync(Y, st);
    if (exch) cudaFreeAsync(exch, st);
    if (psd_dev) cudaFreeAsync(psd_dev, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // host injection table consumed
    if (e != cudaSuccess)
        return set_err(e == cudaErrorMemoryAllocation ? MF_ENOMEM : MF_ECUDA, "synth_segment: %s",
                       cudaGetErrorString(e));
    return MF_OK;
}

// ---------------------------------------------------------------------------
// refinement
// ---------------------------------------------------------------------------
extern "C" int mf_refine_triggers(mf_segment seg, const mf_bank_params *params, const double *theta, int64_t n,
                                  const int64_t *band, double *obj, double *grad, void *cuda_stream) {
    NvtxRange nvtx("mf_refine_triggers");
    if (!seg || !theta || !obj || !grad) return set_err(MF_EINVAL, "NULL argument");
    if (n < 0) return set_err(MF_EINVAL, "n < 0");
    if (n == 0) return MF_OK;
    mf_bank_params p = params ? *params : default_params();
    int rc = check_params(p);
    if (rc) return rc;
    int r0 = ensure_device_init();
    if (r0) return r0;
    int cur = 0;
    MF_CUDA(cudaGetDevice(&cur));
    if (seg->device != cur) return set_err(MF_EINVAL, "segment lives on device %d, current device is %d", seg->device, cur);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const SegDev sd = seg_dev(seg);
    const int bpr = refine_blocks_for(n, sm_count());
    double *partial = nullptr;
    cudaError_t e = dev_malloc_async(&partial, refine_scratch_bytes(n, bpr), st);
    if (e == cudaSuccess) e = launch_refine(sd, p.f_low, p.phase_mode, theta, n, band, obj, grad, partial, bpr, st);
    if (e == cudaSuccess) count_launches(refine_launches(n));
    if (partial) cudaFreeAsync(partial, st);
    if (e != cudaSuccess)
        return set_err(e == cudaErrorMemoryAllocation ? MF_ENOMEM : MF_ECUDA, "refine_triggers: %s",
                       cudaGetErrorString(e));
    return MF_OK;
}

extern "C" int mf_refine_triggers_multi(const mf_segment *segs, int n_seg, const int32_t *row_seg,
                                        const mf_bank_params *params, const double *theta, int64_t n,
                                        const int64_t *band, double *obj, double *grad, void *cuda_stream) {
    if (!segs || !row_seg || !theta || !obj || !grad) return set_err(MF_EINVAL, "NULL argument");
    if (n_seg < 1 || n_seg > kRefineMaxSegs)
        return set_err(MF_EINVAL, "n_seg = %d outside [1, %d]", n_seg, kRefineMaxSegs);
    if (n < 0) return set_err(MF_EINVAL, "n < 0");
    if (n == 0) return MF_OK;
    mf_bank_params p = params ? *params : default_params();
    int rc = check_params(p);
    if (rc) return rc;
    int r0 = ensure_device_init();
    if (r0) return r0;
    int cur = 0;
    cudaGetDevice(&cur);
    std::vector<SegDev> sd((size_t)n_seg);
    for (int s = 0; s < n_seg; ++s) {
        if (!segs[s]) return set_err(MF_EINVAL, "segs[%d] is NULL", s);
        if (segs[s]->device != cur) return set_err(MF_EINVAL, "segs[%d] lives on device %d", s, segs[s]->device);
        sd[(size_t)s] = seg_dev(segs[s]);
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int bpr = refine_blocks_for(n, sm_count());
    double *partial = nullptr;
    cudaError_t e = dev_malloc_async(&partial, refine_scratch_bytes(n, bpr), st);
    if (e == cudaSuccess)
        e = launch_refine_multi(sd.data(), n_seg, row_seg, p.f_low, p.phase_mode, theta, n, band, obj, grad, partial,
                                bpr, st);
    if (e == cudaSuccess) count_launches(refine_launches(n));
    if (partial) cudaFreeAsync(partial, st);
    if (e != cudaSuccess)
        return set_err(e == cudaErrorMemoryAllocation ? MF_ENOMEM : MF_ECUDA, "refine_triggers_multi: %s",
                       cudaGetErrorString(e));
    return MF_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free refinement.  Some callers cannot allocate device memory at
// the point where they refine triggers: an ascent loop that runs while another
// component owns the device allocator, or code that must never trigger an
// allocator call inside its hot loop.  This variant keeps the per-block
// partial sums and row records in a fixed array in device global memory
// instead of the stream allocation that mf_refine_triggers makes.
// ---------------------------------------------------------------------------
static constexpr int64_t kRefineStaticRows = 4096;   // at most this many theta rows per call
static constexpr int kRefineStaticBpr = 16;           // blocks per row (== refine_blocks_per_row())
// 4096 rows x (16 blocks x 8 partial sums x 8 bytes + a 128-byte row record) = 4.5 MiB on every device
// that loads the library
static __device__ __align__(256) double
    g_refine_scratch[kRefineStaticRows * (kRefineStaticBpr * 8 + kRefRowBytesMax / sizeof(double))];

// Device address of g_refine_scratch per device ordinal.  In host code the
// array's name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress once per device, with that device current.
static int refine_scratch_ptr(double **out) {
    static std::mutex mu;
    static std::vector<double *> ptrs;
    int dev = 0;
    MF_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if ((int)ptrs.size() <= dev) ptrs.resize((size_t)dev + 1, nullptr);
    if (!ptrs[(size_t)dev]) {
        void *p = nullptr;
        MF_CUDA(cudaGetSymbolAddress(&p, g_refine_scratch));
        ptrs[(size_t)dev] = (double *)p;
    }
    *out = ptrs[(size_t)dev];
    return MF_OK;
}

extern "C" int mf_refine_triggers_static(mf_segment seg, const mf_bank_params *params, const double *theta, int64_t n,
                                         const int64_t *band, double *obj, double *grad, void *cuda_stream) {
    if (!seg || !theta || !obj || !grad) return set_err(MF_EINVAL, "NULL argument");
    if (n < 0) return set_err(MF_EINVAL, "n < 0");
    if (n > kRefineStaticRows)
        return set_err(MF_EINVAL, "n = %lld exceeds the fixed scratch of %lld rows of mf_refine_triggers_static",
                       (long long)n, (long long)kRefineStaticRows);
    if (refine_blocks_per_row() != kRefineStaticBpr) return set_err(MF_ENOTSUP, "scratch layout mismatch");
    if (n == 0) return MF_OK;
    mf_bank_params p = params ? *params : default_params();
    int rc = check_params(p);
    if (rc) return rc;
    rc = ensure_device_init();
    if (rc) return rc;
    int cur = 0;
    MF_CUDA(cudaGetDevice(&cur));
    if (seg->device != cur) return set_err(MF_EINVAL, "segment lives on device %d, current device is %d", seg->device, cur);
    double *scratch = nullptr;
    rc = refine_scratch_ptr(&scratch);
    if (rc) return rc;
    // every partial sum the final kernel reads is written by the first kernel of
    // the same call, so nothing in the scratch needs clearing
    const SegDev sd = seg_dev(seg);
    MF_CUDA(launch_refine(sd, p.f_low, p.phase_mode, theta, n, band, obj, grad, scratch, kRefineStaticBpr,
                          (cudaStream_t)cuda_stream));
    count_launches(refine_launches(n));
    return MF_OK;
}

extern "C" int mf_debug_fail_alloc(int64_t countdown) {
    g_fail_alloc.store(countdown < 0 ? -1 : countdown);
    return MF_OK;
}
