// mf_events.cu -- events from triggers, and the chi^2 of Eq. (5) at single
// samples.
//
// Clustering (the paper reports events, Sec. 3.3, and gives no rule): single
// linkage in time with a maximum gap of `window` samples, first over the
// triggers of each (template, segment) pair (input sorted by (tmpl, seg, j)),
// then over those clusters' loudest members of all templates within a
// segment (re-sorted by (seg, j, tmpl)).  A cluster's representative is its
// loudest member, the earliest in the pass's order on ties.  Each pass is
//   start flags -> inclusive scan (cluster ids) -> packed atomicMax of
//   (rho bits, ~index) and member counts per cluster -> emit,
// with the record count read on the device, so the host never synchronises.
//
// chi^2 at a sample (Eq. 5 at t = j dt): the sub-band sums of Eq. (1),
//   R_l = sum_{k in [b_l, b_{l+1})} W_k e^{-i Psi_k} e^{2 pi i j k / N},
//   chi^2 = p (P_tot/Q) sum_l |R_l - R/p|^2,  R = sum_l R_l,
// with the sub-band edges of mf_chisq_series and the filter's phase form
// (FP64 anchors, FP32 quartic Taylor, FP32 sincos); (j k mod N) is exact in
// integers.  One row per point, blocks over the band, FP64 block totals per
// sub-band in a fixed order.
#include "mf_filter.cuh"
#include "mf_tmpl.cuh"

namespace mf {

// ---------------------------------------------------------------------------
// device-wide inclusive scan of uint32 flags (n read on the device)
// ---------------------------------------------------------------------------
constexpr int kSuThreads = 256, kSuPer = 8, kSuBlock = kSuThreads * kSuPer;

__device__ __forceinline__ int64_t dev_count(const int64_t *cnt, int64_t cap) {
    const int64_t n = *cnt;
    return n < cap ? (n > 0 ? n : 0) : cap;
}

__global__ void k_su_local(const uint32_t *__restrict__ in, const int64_t *cnt, int64_t cap, uint32_t *__restrict__ out,
                           uint32_t *__restrict__ bsum) {
    __shared__ uint32_t ws[kSuThreads / 32];
    const int64_t n = dev_count(cnt, cap);
    const int64_t base = (int64_t)blockIdx.x * kSuBlock + (int64_t)threadIdx.x * kSuPer;
    uint32_t v[kSuPer], run = 0;
#pragma unroll
    for (int e = 0; e < kSuPer; ++e) {
        v[e] = (base + e < n) ? in[base + e] : 0u;
        run += v[e];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    uint32_t wo = 0;
    for (int w = 0; w < warp; ++w) wo += ws[w];
    uint32_t acc = wo + incl - run;
#pragma unroll
    for (int e = 0; e < kSuPer; ++e) {
        acc += v[e];
        if (base + e < n) out[base + e] = acc;
    }
    if (threadIdx.x == kSuThreads - 1) bsum[blockIdx.x] = wo + incl;
}

// exclusive scan of the block totals by one block, chunk by chunk
__global__ void k_su_sums(uint32_t *bsum, int nb) {
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c0 = 0; c0 < nb; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        const uint32_t x = i < nb ? bsum[i] : 0u;
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) ws[warp] = incl;
        __syncthreads();
        uint32_t wo = 0;
        for (int w = 0; w < warp; ++w) wo += ws[w];
        const uint32_t c = carry;
        if (i < nb) bsum[i] = c + wo + incl - x;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = c + wo + incl;
        __syncthreads();
    }
}

__global__ void k_su_add(uint32_t *out, const int64_t *cnt, int64_t cap, const uint32_t *__restrict__ bsum) {
    const int64_t n = dev_count(cnt, cap);
    const int64_t base = (int64_t)blockIdx.x * kSuBlock;
    const uint32_t add = bsum[blockIdx.x];
    for (int e = threadIdx.x; e < kSuBlock; e += kSuThreads)
        if (base + e < n) out[base + e] += add;
}

static int su_blocks(int64_t cap) { return (int)((cap + kSuBlock - 1) / kSuBlock); }

static cudaError_t launch_scan_u32(const uint32_t *in, const int64_t *cnt, int64_t cap, uint32_t *out, uint32_t *bsum,
                                   cudaStream_t st) {
    const int nb = su_blocks(cap);
    k_su_local<<<nb, kSuThreads, 0, st>>>(in, cnt, cap, out, bsum);
    k_su_sums<<<1, 1024, 0, st>>>(bsum, nb);
    k_su_add<<<nb, kSuThreads, 0, st>>>(out, cnt, cap, bsum);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// clustering passes
// ---------------------------------------------------------------------------
// mode 1: same (tmpl, seg); mode 2: same seg.  Also clears the per-cluster
// accumulators (a cluster id never exceeds the index of its first member).
__global__ void k_cl_start(const mf_trigger *__restrict__ t, const int64_t *cnt, int64_t cap, int window, int mode,
                           uint32_t *__restrict__ flag, unsigned long long *__restrict__ best,
                           uint32_t *__restrict__ members, uint32_t *__restrict__ weight_sum) {
    const int64_t n = dev_count(cnt, cap);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t f = 1u;
        if (i > 0) {
            const mf_trigger a = t[i - 1], b = t[i];
            const bool same = mode == 1 ? (a.tmpl == b.tmpl && a.seg == b.seg) : (a.seg == b.seg);
            f = (same && (int64_t)b.j - (int64_t)a.j <= window) ? 0u : 1u;
        }
        flag[i] = f;
        best[i] = 0ull;
        members[i] = 0u;
        if (weight_sum) weight_sum[i] = 0u;
    }
}

// weights: NULL (each record counts 1) or per-record counts reached through perm
__global__ void k_cl_reduce(const mf_trigger *__restrict__ t, const int64_t *cnt, int64_t cap,
                            const uint32_t *__restrict__ incl, unsigned long long *best, uint32_t *members,
                            const uint32_t *__restrict__ perm, const uint32_t *__restrict__ weights,
                            uint32_t *weight_sum) {
    const int64_t n = dev_count(cnt, cap);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = incl[i] - 1u;
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(fmaxf(t[i].rho, 0.f)) << 32) | (0xffffffffull - (unsigned long long)i);
        atomicMax(&best[c], key);
        atomicAdd(&members[c], 1u);
        if (weights) atomicAdd(&weight_sum[c], weights[perm[i]]);
    }
}

// pass-1 output: the clusters' representatives with their trigger counts and
// the (seg, j, tmpl) sort keys; *n_c = the cluster count
__global__ void k_cl_emit1(const mf_trigger *__restrict__ t, const int64_t *cnt, int64_t cap,
                           const uint32_t *__restrict__ incl, const unsigned long long *__restrict__ best,
                           const uint32_t *__restrict__ members, mf_trigger *__restrict__ rep,
                           uint32_t *__restrict__ rep_count, uint64_t *__restrict__ keys, KeyLayout kl,
                           int64_t *n_c) {
    const int64_t n = dev_count(cnt, cap);
    const int64_t nc = n > 0 ? (int64_t)incl[n - 1] : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_c = nc;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t idx = (int64_t)(0xffffffffull - (best[c] & 0xffffffffull));
        const mf_trigger r = t[idx];
        rep[c] = r;
        rep_count[c] = members[c];
        keys[c] = ((uint64_t)r.seg << (kl.j_bits + kl.tmpl_bits)) | ((uint64_t)r.j << kl.tmpl_bits) | (uint64_t)r.tmpl;
    }
}

__global__ void k_cl_emit2(const mf_trigger *__restrict__ t, const int64_t *cnt, int64_t cap,
                           const uint32_t *__restrict__ incl, const unsigned long long *__restrict__ best,
                           const uint32_t *__restrict__ members, const uint32_t *__restrict__ weight_sum,
                           mf_event *__restrict__ ev, int64_t ev_cap, int64_t *n_events, int *status) {
    const int64_t n = dev_count(cnt, cap);
    const int64_t nc = n > 0 ? (int64_t)incl[n - 1] : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *n_events = nc;
        if (nc > ev_cap) atomicOr(status, 1);
    }
    const int64_t m = nc < ev_cap ? nc : ev_cap;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < m; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t idx = (int64_t)(0xffffffffull - (best[c] & 0xffffffffull));
        const mf_trigger r = t[idx];
        mf_event e;
        e.tmpl = r.tmpl;
        e.seg = r.seg;
        e.j = r.j;
        e.rho = r.rho;
        e.z_re = r.z_re;
        e.z_im = r.z_im;
        e.n_trig = (int32_t)weight_sum[c];
        e.n_tmpl = (int32_t)members[c];
        ev[c] = e;
    }
}

cudaError_t launch_cluster(const mf_trigger *trig, const int64_t *n_trig, int64_t cap, int window, KeyLayout kl,
                           ClusterScratch &w, mf_event *events, int64_t ev_cap, int64_t *n_events, int n_sm,
                           int64_t spin_limit, cudaStream_t st) {
    const int grid = 4 * n_sm, thr = 256;
    cudaError_t e;
    // pass 1: per (template, segment)
    k_cl_start<<<grid, thr, 0, st>>>(trig, n_trig, cap, window, 1, w.flag, w.best, w.members, nullptr);
    if ((e = launch_scan_u32(w.flag, n_trig, cap, w.incl, w.bsum, st)) != cudaSuccess) return e;
    k_cl_reduce<<<grid, thr, 0, st>>>(trig, n_trig, cap, w.incl, w.best, w.members, nullptr, nullptr, nullptr);
    k_cl_emit1<<<grid, thr, 0, st>>>(trig, n_trig, cap, w.incl, w.best, w.members, w.rep, w.rep_count, w.keys, kl,
                                     w.n_c);
    // re-order the representatives by (seg, j, tmpl)
    const int key_bits = kl.j_bits + kl.seg_bits + kl.tmpl_bits;
    e = launch_sort_triggers((const unsigned long long *)w.n_c, cap, key_bits, w.rep, w.keys, w.keys_tmp, w.idx_a,
                             w.idx_b, w.ghist, w.tstat, w.tickets, w.sorted, w.perm, w.n_sorted, w.status, n_sm,
                             spin_limit, st);
    if (e != cudaSuccess) return e;
    // pass 2: across templates within a segment
    k_cl_start<<<grid, thr, 0, st>>>(w.sorted, w.n_c, cap, window, 2, w.flag, w.best, w.members, w.wsum);
    if ((e = launch_scan_u32(w.flag, w.n_c, cap, w.incl, w.bsum, st)) != cudaSuccess) return e;
    k_cl_reduce<<<grid, thr, 0, st>>>(w.sorted, w.n_c, cap, w.incl, w.best, w.members, w.perm, w.rep_count, w.wsum);
    k_cl_emit2<<<grid, thr, 0, st>>>(w.sorted, w.n_c, cap, w.incl, w.best, w.members, w.wsum, events, ev_cap,
                                     n_events, w.status);
    return cudaGetLastError();
}

int cluster_launches(int key_bits) { return 2 * (4 + 3) + sort_launches(key_bits); }
int64_t cluster_scan_blocks(int64_t cap) { return su_blocks(cap); }

// ---------------------------------------------------------------------------
// chi^2 at single samples
// ---------------------------------------------------------------------------
constexpr int kCpThreads = 256;
constexpr int kCpAnchors = kCpThreads;

struct CpRow {
    double c[4];
    int64_t b[kChisqMaxBands + 1];
    double pratio;
    uint32_t j;
    int log2D, valid;
};

__device__ void cp_row_setup(const SegDev &seg, const double *tmpl, int n_t, double f_low, int anchored, int t,
                             int32_t j, int p, CpRow &r) {
    r.valid = (t >= 0 && t < n_t && j >= 0 && (int64_t)j < seg.N) ? 1 : 0;
    const double *T = tmpl + (int64_t)(r.valid ? t : 0) * kTmplStride;
    r.c[0] = T[TF_C1]; r.c[1] = T[TF_C2]; r.c[2] = T[TF_C3]; r.c[3] = T[TF_C5];
    const double N = (double)seg.N, fs = seg.fs;
    const double fc = T[TF_FISCO] < 0.5 * fs ? T[TF_FISCO] : 0.5 * fs;
    int64_t lo = (int64_t)ceil(f_low * N / fs), hi = (int64_t)floor(fc * N / fs) + 1;
    if (lo < 1) lo = 1;
    if (hi > seg.N / 2) hi = seg.N / 2;
    if (hi < lo || !r.valid) hi = lo;
    const double Q = seg.P[hi] - seg.P[lo];
    r.pratio = Q > 0.0 ? seg.consts->P_tot / Q : 0.0;
    r.b[0] = lo;
    r.b[p] = hi;
    r.j = (uint32_t)(r.valid ? j : 0);
    r.log2D = 0;
    if (anchored) {
        const double f0 = (double)lo * seg.df;
        r.log2D = anchor_log2D(psi_deriv_bound_u(r.c, f0, 1), psi_deriv_bound_u(r.c, f0, 5), seg.df);
    }
}

// interior sub-band edges, one thread per edge: the rule and arithmetic of k_chisq_units
__device__ void cp_row_edges(const SegDev &seg, int p, CpRow &r) {
    const int l = threadIdx.x;
    if (l < 1 || l >= p) return;
    const int64_t lo = r.b[0], hi = r.b[p];
    const double P0 = seg.P[lo], Q = seg.P[hi] - P0;
    const double target = ((double)l / (double)p) * Q;
    int64_t a = lo, c = hi;
    while (a < c) {
        const int64_t m = a + ((c - a) >> 1);
        if (seg.P[m] - P0 >= target) c = m;
        else a = m + 1;
    }
    r.b[l] = a;
}

template <int NS>
struct CpSegs {
    SegDev s[NS];
    int n;
};

// partial[(row * bpr + block) * p + l] = (re, im) of R_l over this block's bins
template <int NS>
__global__ void __launch_bounds__(kCpThreads)
    k_chisq_points(const __grid_constant__ CpSegs<NS> segs, const double *__restrict__ tmpl, int n_t, double f_low,
                   int anchored, const int32_t *__restrict__ rows, int64_t stride, int p, double2 *__restrict__ partial) {
    __shared__ CpRow row;
    __shared__ float4 sanc[kCpAnchors];
    __shared__ float sanc4[kCpAnchors];
    __shared__ double red[2][kCpThreads / 32];
    const int64_t i = blockIdx.y;
    const int32_t t = rows[i * stride], sg = rows[i * stride + 1], jj = rows[i * stride + 2];
    const bool seg_ok = sg >= 0 && sg < segs.n;
    const SegDev &seg = segs.s[seg_ok ? sg : 0];
    if (threadIdx.x == 0) {
        cp_row_setup(seg, tmpl, n_t, f_low, anchored, t, jj, p, row);
        if (!seg_ok) {
            row.valid = 0;
            row.b[p] = row.b[0];
        }
    }
    __syncthreads();
    cp_row_edges(seg, p, row);
    __syncthreads();
    const uint32_t nmask = (uint32_t)(seg.N - 1);
    const int64_t k_lo = row.b[0], k_hi = row.b[p];
    // this block's bin range: whole anchor groups (or a plain chunk in the FP64 form)
    const int lg = row.log2D > 0 ? row.log2D : 8;
    const int64_t g_lo = k_lo >> lg, g_hi = k_hi > k_lo ? ((k_hi - 1) >> lg) : g_lo - 1;
    const int64_t ng = g_hi - g_lo + 1;
    const int64_t gpb = (ng + gridDim.x - 1) / gridDim.x;
    const int64_t gb0 = g_lo + (int64_t)blockIdx.x * gpb;
    const int64_t gb1 = (gb0 + gpb < g_lo + ng) ? gb0 + gpb : g_lo + ng;
    int64_t r0 = gb0 << lg, r1 = gb1 << lg;
    if (r0 < k_lo) r0 = k_lo;
    if (r1 > k_hi) r1 = k_hi;
    const float invN = 1.0f / (float)seg.N;
    const int half = (1 << lg) >> 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double2 *out = partial + ((int64_t)i * gridDim.x + blockIdx.x) * p;
    for (int l = 0; l < p; ++l) {
        int64_t a = row.b[l] > r0 ? row.b[l] : r0, b = row.b[l + 1] < r1 ? row.b[l + 1] : r1;
        float sr = 0.f, si = 0.f;
        // anchors of the groups this sub-band slice touches, in chunks of kCpAnchors
        for (int64_t k0 = a; k0 < b;) {
            const int64_t ga = k0 >> lg;
            int64_t ge = ga + kCpAnchors;
            int64_t kend = ge << lg;
            if (kend > b) kend = b;
            if (row.log2D > 0) {
                const int64_t gend = ((kend - 1) >> lg) + 1;
                if (ga + threadIdx.x < gend)
                    anchor_record(row.c[0], row.c[1], row.c[2], row.c[3], ga + threadIdx.x, lg, seg.df,
                                  sanc[threadIdx.x], sanc4[threadIdx.x]);
                __syncthreads();
            }
            for (int64_t k = k0 + threadIdx.x; k < kend; k += kCpThreads) {
                float psi;
                if (row.log2D > 0) {
                    const int ai = (int)((k >> lg) - ga);
                    const float4 an = sanc[ai];
                    const float d = (float)(int)((k & ((1 << lg) - 1)) - half);
                    psi = an.x + d * (an.y + d * (an.z + d * (an.w + d * sanc4[ai])));
                } else {
                    const double f = (double)k * seg.df;
                    double u = (double)rcbrtf((float)f);
                    u = u * (4.0 - f * u * u * u) * (1.0 / 3.0);
                    double ps = -0.125 + u * (row.c[0] + u * (row.c[1] + u * (row.c[2] + u * u * row.c[3])));
                    psi = (float)(ps - rint(ps));
                }
                float ph = (float)(((uint32_t)k * row.j) & nmask) * invN - psi;
                ph -= rintf(ph);
                float sn, cs;
                __sincosf(6.283185307179586f * ph, &sn, &cs);
                const float2 w = __ldg(&seg.W[k]);
                sr += w.x * cs - w.y * sn;
                si += w.x * sn + w.y * cs;
            }
            if (row.log2D > 0) __syncthreads();
            k0 = kend;
        }
        // block totals of this sub-band (FP64, fixed order)
        double vr = sr, vi = si;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vr += __shfl_xor_sync(0xffffffffu, vr, o);
            vi += __shfl_xor_sync(0xffffffffu, vi, o);
        }
        if (lane == 0) { red[0][warp] = vr; red[1][warp] = vi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double tr = 0.0, ti = 0.0;
            for (int w = 0; w < kCpThreads / 32; ++w) { tr += red[0][w]; ti += red[1][w]; }
            out[l] = make_double2(tr, ti);
        }
        __syncthreads();
    }
}

template <int NS>
__global__ void k_chisq_points_final(const __grid_constant__ CpSegs<NS> segs, const double *__restrict__ tmpl,
                                     int n_t, double f_low, const int32_t *__restrict__ rows, int64_t stride, int p,
                                     const double2 *__restrict__ partial, int bpr, int64_t n,
                                     float *__restrict__ chisq) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t t = rows[i * stride], sg = rows[i * stride + 1], jj = rows[i * stride + 2];
    const bool seg_ok = sg >= 0 && sg < segs.n;
    if (!seg_ok || t < 0 || t >= n_t || jj < 0 || (int64_t)jj >= segs.s[sg].N) {
        chisq[i] = __int_as_float(0x7fc00000);
        return;
    }
    const SegDev &seg = segs.s[sg];
    const double *T = tmpl + (int64_t)t * kTmplStride;
    const double N = (double)seg.N, fs = seg.fs;
    const double fc = T[TF_FISCO] < 0.5 * fs ? T[TF_FISCO] : 0.5 * fs;
    int64_t lo = (int64_t)ceil(f_low * N / fs), hi = (int64_t)floor(fc * N / fs) + 1;
    if (lo < 1) lo = 1;
    if (hi > seg.N / 2) hi = seg.N / 2;
    if (hi < lo) hi = lo;
    const double Q = seg.P[hi] - seg.P[lo];
    const double pratio = Q > 0.0 ? seg.consts->P_tot / Q : 0.0;
    double Rr = 0.0, Ri = 0.0;
    for (int l = 0; l < p; ++l)
        for (int b = 0; b < bpr; ++b) {
            const double2 v = partial[((int64_t)i * bpr + b) * p + l];
            Rr += v.x;
            Ri += v.y;
        }
    double s = 0.0;
    for (int l = 0; l < p; ++l) {
        double lr = 0.0, li = 0.0;
        for (int b = 0; b < bpr; ++b) {
            const double2 v = partial[((int64_t)i * bpr + b) * p + l];
            lr += v.x;
            li += v.y;
        }
        const double dr = lr - Rr / p, di = li - Ri / p;
        s += dr * dr + di * di;
    }
    chisq[i] = (float)((double)p * pratio * s);
}

cudaError_t launch_chisq_points(const SegDev *segs, int n_seg, const double *tmpl, int n_t, double f_low,
                                int phase_mode, const int32_t *rows, int64_t stride, int64_t n, int p, int bpr,
                                double2 *partial, float *chisq, cudaStream_t st) {
    if (n_seg < 1 || n_seg > kRefineMaxSegs || p < 1 || p > kChisqMaxBands) return cudaErrorInvalidValue;
    const int anchored = phase_mode == MF_PHASE_FP64 ? 0 : 1;
    CpSegs<kRefineMaxSegs> tab;
    for (int s = 0; s < n_seg; ++s) tab.s[s] = segs[s];
    tab.n = n_seg;
    k_chisq_points<kRefineMaxSegs><<<dim3((unsigned)bpr, (unsigned)n), kCpThreads, 0, st>>>(
        tab, tmpl, n_t, f_low, anchored, rows, stride, p, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_chisq_points_final<kRefineMaxSegs><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(tab, tmpl, n_t, f_low, rows,
                                                                                      stride, p, partial, bpr, n,
                                                                                      chisq);
    return cudaGetLastError();
}

}  // namespace mf
