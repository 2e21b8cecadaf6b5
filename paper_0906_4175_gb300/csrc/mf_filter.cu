// mf_filter.cu -- the hot path of the bank filter (Eqs. 1, 3, 4 of
// arXiv:0906.4175): per (template, segment) unit
//   k_units    band [k_lo, k_hi) (Sec. 1.1 band rule), sigma from the FP64
//              prefix table, rho and z scale factors, anchor range;
//   k_anchors  the 2PN phase Psi/(2 pi) in FP64 at anchor bins, reduced mod 1,
//              plus its first four k-derivatives (FP32 Taylor coefficients);
//   pass 1     template generation h~_k = e^{-i Psi_k} in registers (FP32
//              quartic Taylor from the nearest anchor, __sincosf of the reduced
//              phase), weighting by W_k = f^(-7/6) conj(s~_k)/S_k, column IFFTs,
//              four-step twiddle, one complex64 exchange write;
//   pass 2     row IFFTs and the rho epilogue: |z|^2 threshold test, argmax with
//              lowest-j tie-break, warp-aggregated trigger append;
//   k_reduce_peaks / k_sort_triggers   deterministic peaks and (tmpl, seg, j)
//              ordered triggers.
// Neither h~(f) nor z(t) is written to memory.
#include "mf_filter.cuh"

namespace mf {

// ---------------------------------------------------------------------------
// per-unit set-up
// ---------------------------------------------------------------------------
__global__ void k_units(SegDev seg, const double *__restrict__ tmpl, int n_t, double f_low, float thr,
                        int log2D, UnitInfo *__restrict__ units) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_t) return;
    const double *T = tmpl + (int64_t)t * kTmplStride;
    const double N = (double)seg.N, fs = seg.fs;
    const double fisco = T[TF_FISCO];
    const double fc = fisco < 0.5 * fs ? fisco : 0.5 * fs;
    int64_t lo = (int64_t)ceil(f_low * N / fs);
    int64_t hi = (int64_t)floor(fc * N / fs) + 1;
    if (lo < 1) lo = 1;
    if (hi > seg.N / 2) hi = seg.N / 2;
    if (hi < lo) hi = lo;
    const double Q = seg.P[hi] - seg.P[lo];              // sum_band f^(-7/3)/S  (Eq. 4 / (4 df A^2))
    const double rs = sqrt(seg.consts->P_tot / Q);
    UnitInfo u;
    u.k_lo = (int32_t)lo;
    u.k_hi = (int32_t)hi;
    u.g_lo = (int32_t)(lo >> log2D);
    u.n_anc = (int32_t)(((hi - 1) >> log2D) - (lo >> log2D) + 1);
    u.rho_scale = (float)rs;
    const double th = (double)thr / rs;
    u.thr2 = (float)(th * th);
    u.z_scale = (float)(4.0 * seg.df * T[TF_AMP] / seg.consts->alpha);
    u.tmpl = t;
    units[t] = u;
}

__global__ void k_anchors(SegDev seg, const double *__restrict__ tmpl, const UnitInfo *__restrict__ units,
                          int unit0, int log2D, int max_anc, float4 *__restrict__ anchors,
                          float *__restrict__ anchors4) {
    const int b = blockIdx.y;
    const UnitInfo u = units[unit0 + b];
    const double *T = tmpl + (int64_t)u.tmpl * kTmplStride;
    const double c1 = T[TF_C1], c2 = T[TF_C2], c3 = T[TF_C3], c5 = T[TF_C5];
    float4 *out = anchors + (int64_t)b * max_anc;
    float *out4 = anchors4 + (int64_t)b * max_anc;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < u.n_anc; i += gridDim.x * blockDim.x) {
        float4 r;
        float r4;
        anchor_record(c1, c2, c3, c5, (int64_t)u.g_lo + i, log2D, seg.df, r, r4);
        out[i] = r;
        out4[i] = r4;
    }
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------
cudaError_t launch_units(const SegDev &seg, const double *tmpl, int n_t, double f_low, float thr, int log2D,
                         UnitInfo *units, cudaStream_t st) {
    k_units<<<(n_t + 255) / 256, 256, 0, st>>>(seg, tmpl, n_t, f_low, thr, log2D, units);
    return cudaGetLastError();
}

cudaError_t launch_anchors(const SegDev &seg, const double *tmpl, const UnitInfo *units, int unit0, int n_units,
                           int log2D, int max_anc, float4 *anchors, float *anchors4, cudaStream_t st) {
    const int per = 256;
    int gx = (max_anc + per - 1) / per;
    if (gx > 64) gx = 64;
    k_anchors<<<dim3(gx, n_units), per, 0, st>>>(seg, tmpl, units, unit0, log2D, max_anc, anchors, anchors4);
    return cudaGetLastError();
}

namespace {
struct Pass1Op {
    const SegDev &seg;
    const UnitInfo *units;
    int unit0, n_units, log2D, max_anc, phase_mode;
    const float4 *anchors;
    const float *anchors4;
    float2 *exch;
    const double *tmpl;
    cudaStream_t st;
    template <int N2, int N1>
    cudaError_t run() {
        constexpr int C = seqs_per_cta<N2>(N1);
        typename ExchSink<N2, C, +1, cx_ilog2(N1)>::Params kp{exch, seg.log2N1, seg.log2N};
        const dim3 grid(N1 / C, n_units);
        if (phase_mode == MF_PHASE_FP32) {
            typename TemplateSrcF32<N2, C, cx_ilog2(N1)>::Params sp{seg.W, units, tmpl, (float)seg.df};
            return run_pass<N2, C, true, +1, TemplateSrcF32<N2, C, cx_ilog2(N1)>, ExchSink<N2, C, +1, cx_ilog2(N1)>>(grid, sp, kp, st, unit0);
        }
        typename TemplateSrc<N2, C, cx_ilog2(N1)>::Params sp{seg.W, units, anchors, anchors4, max_anc, log2D};
        return run_pass<N2, C, true, +1, TemplateSrc<N2, C, cx_ilog2(N1)>, ExchSink<N2, C, +1, cx_ilog2(N1)>>(grid, sp, kp, st, unit0);
    }
};

struct Pass2Op {
    const SegDev &seg;
    const UnitInfo *units;
    int unit0, n_units;
    const float2 *exch;
    float4 *partials;
    int seg_idx;
    KeyLayout kl;
    mf_trigger *staged;
    uint64_t *keys;
    unsigned long long *counter;
    int64_t cap;
    cudaStream_t st;
    template <int N2, int N1>
    cudaError_t run() {
        constexpr int C = seqs_per_cta<N1>(N2);
        const int nblk = N2 / C;
        typename RowSrc<N1, C>::Params sp{exch, seg.log2N1, seg.log2N};
        typename RhoSink<N1, C>::Params kp{units, partials, staged, keys, counter, cap,
                                           seg.log2N2, nblk, seg_idx, kl};
        return run_pass<N1, C, false, +1, RowSrc<N1, C>, RhoSink<N1, C>>(dim3(nblk, n_units), sp, kp, st, unit0);
    }
};

struct BlocksOp {
    int nblk = 0;
    template <int N2, int N1>
    cudaError_t run() {
        nblk = N2 / seqs_per_cta<N1>(N2);
        return cudaSuccess;
    }
};

struct AttrOp {
    template <int N2, int N1>
    cudaError_t run() {
        constexpr int C1 = seqs_per_cta<N2>(N1);
        constexpr int C2 = seqs_per_cta<N1>(N2);
        cudaError_t e;
        if ((e = set_pass_attrs<N2, C1, true, +1, TemplateSrc<N2, C1, cx_ilog2(N1)>, ExchSink<N2, C1, +1, cx_ilog2(N1)>>())) return e;
        if ((e = set_pass_attrs<N2, C1, true, +1, TemplateSrcF32<N2, C1, cx_ilog2(N1)>, ExchSink<N2, C1, +1, cx_ilog2(N1)>>())) return e;
        return set_pass_attrs<N1, C2, false, +1, RowSrc<N1, C2>, RhoSink<N1, C2>>();
    }
};
}  // namespace

cudaError_t launch_pass1(const SegDev &seg, const UnitInfo *units, int unit0, int n_units, int log2D, int max_anc,
                         const float4 *anchors, const float *anchors4, float2 *exch, int phase_mode,
                         const double *tmpl, cudaStream_t st) {
    Pass1Op op{seg, units, unit0, n_units, log2D, max_anc, phase_mode, anchors, anchors4, exch, tmpl, st};
    return dispatch_split(seg.log2N, op);
}

cudaError_t launch_pass2(const SegDev &seg, const UnitInfo *units, int unit0, int n_units, const float2 *exch,
                         float4 *partials, int seg_idx, KeyLayout kl, mf_trigger *staged, uint64_t *keys,
                         unsigned long long *counter, int64_t cap, cudaStream_t st) {
    Pass2Op op{seg, units, unit0, n_units, exch, partials, seg_idx, kl, staged, keys, counter, cap, st};
    return dispatch_split(seg.log2N, op);
}

int pass2_blocks(int log2N) {
    BlocksOp op;
    dispatch_split(log2N, op);
    return op.nblk;
}

cudaError_t filter_kernel_attributes() {
    for (int lg = 10; lg <= 22; ++lg) {
        AttrOp op;
        cudaError_t e = dispatch_split(lg, op);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// peaks: one warp per unit reduces the pass-2 partials of that unit
// ---------------------------------------------------------------------------
__global__ void k_reduce_peaks(const UnitInfo *__restrict__ units, int n_units, const float4 *__restrict__ partials,
                               int nblk, int seg_idx, int n_seg, mf_peak *__restrict__ peaks) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_units) return;
    float bp = -1.f;
    int bj = 0x7fffffff;
    float bx = 0.f, by = 0.f;
    const float4 *pp = partials + (int64_t)warp * nblk;
    for (int i = lane; i < nblk; i += 32) {
        const float4 c = pp[i];
        const int cj = __float_as_int(c.y);
        if (c.x > bp || (c.x == bp && cj < bj)) { bp = c.x; bj = cj; bx = c.z; by = c.w; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float op = __shfl_xor_sync(0xffffffffu, bp, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        const float ox = __shfl_xor_sync(0xffffffffu, bx, o);
        const float oy = __shfl_xor_sync(0xffffffffu, by, o);
        if (op > bp || (op == bp && oj < bj)) { bp = op; bj = oj; bx = ox; by = oy; }
    }
    if (lane == 0) {
        const UnitInfo u = units[warp];
        mf_peak pk;
        pk.rho = sqrtf(bp) * u.rho_scale;
        pk.j = bj;
        pk.z_re = bx * u.z_scale;
        pk.z_im = by * u.z_scale;
        peaks[(int64_t)u.tmpl * n_seg + seg_idx] = pk;
    }
}

cudaError_t launch_reduce_peaks(const SegDev &seg, const UnitInfo *units, int n_units, const float4 *partials,
                                int nblk, int seg_idx, int n_seg, mf_peak *peaks, cudaStream_t st) {
    (void)seg;
    const int threads = 256;
    const int blocks = (n_units * 32 + threads - 1) / threads;
    k_reduce_peaks<<<blocks, threads, 0, st>>>(units, n_units, partials, nblk, seg_idx, n_seg, peaks);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Trigger compaction: stable LSD radix sort of the (tmpl, seg, j) keys by one
// CTA of 32 warps (8-bit digits; warp w owns the w-th contiguous chunk; ranks
// inside a warp by __match_any_sync keep equal digits in input order), then a
// gather into the caller's buffer.  Sets status bit 0 on overflow.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t block_exclusive_scan_1024(uint32_t x, uint32_t *wtot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = wtot[lane], wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        wtot[lane] = wi - w;
    }
    __syncthreads();
    const uint32_t r = wtot[warp] + incl - x;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(1024, 1)
    k_sort_triggers(const unsigned long long *__restrict__ counter, int64_t cap, int key_bits,
                    const mf_trigger *__restrict__ staged, uint64_t *keys, uint64_t *keys_tmp, uint32_t *idx_a,
                    uint32_t *idx_b, mf_trigger *__restrict__ out, int64_t *n_out, int *status) {
    __shared__ uint32_t hist[256][33];
    __shared__ uint32_t wtot[32];
    const unsigned long long total = *counter;
    const int64_t n = (int64_t)(total < (unsigned long long)cap ? total : (unsigned long long)cap);
    if (threadIdx.x == 0) {
        *n_out = (int64_t)total;
        if (total > (unsigned long long)cap) atomicOr(status, 1);
    }
    if (n == 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t chunk = (n + 31) / 32;
    const int64_t lo = (int64_t)warp * chunk;
    const int64_t hi = (lo + chunk < n) ? lo + chunk : n;
    const int npass = key_bits > 0 ? (key_bits + 7) / 8 : 1;
    const uint64_t *kin = keys;
    const uint32_t *iin = nullptr;
    uint64_t *kbuf[2] = {keys_tmp, keys};
    uint32_t *ibuf[2] = {idx_a, idx_b};
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int pass = 0; pass < npass; ++pass) {
        uint64_t *kout = kbuf[pass & 1];
        uint32_t *iout = ibuf[pass & 1];
        const int shift = 8 * pass;
        for (int e = threadIdx.x; e < 256 * 32; e += 1024) hist[e >> 5][e & 31] = 0u;
        __syncthreads();
        if (lo < hi)
            for (int64_t i = lo + lane; i < hi; i += 32) atomicAdd(&hist[(kin[i] >> shift) & 255u][warp], 1u);
        __syncthreads();
        uint32_t loc[8], s = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = threadIdx.x * 8 + q;
            loc[q] = s;
            s += hist[e >> 5][e & 31];
        }
        const uint32_t off = block_exclusive_scan_1024(s, wtot);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = threadIdx.x * 8 + q;
            hist[e >> 5][e & 31] = off + loc[q];
        }
        __syncthreads();
        for (int64_t base = lo; base < hi; base += 32) {
            const int64_t i = base + lane;
            const bool act = i < hi;
            const uint64_t key = act ? kin[i] : 0ull;
            const uint32_t id = act ? (iin ? iin[i] : (uint32_t)i) : 0u;
            const uint32_t d = act ? (uint32_t)((key >> shift) & 255u) : (256u + (uint32_t)lane);
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const int rank = __popc(peers & lt_mask);
            if (act) {
                const uint32_t pos = hist[d][warp] + (uint32_t)rank;
                kout[pos] = key;
                iout[pos] = id;
            }
            __syncwarp();
            if (act && rank == 0) hist[d][warp] += (uint32_t)__popc(peers);
            __syncwarp();
        }
        __syncthreads();
        kin = kout;
        iin = iout;
    }
    for (int64_t i = threadIdx.x; i < n; i += 1024) out[i] = staged[iin[i]];
}

cudaError_t launch_sort_triggers(const unsigned long long *counter, int64_t cap, int key_bits,
                                 const mf_trigger *staged, const uint64_t *keys, uint64_t *keys_tmp,
                                 uint32_t *idx_a, uint32_t *idx_b, mf_trigger *out, int64_t *n_out, int *status,
                                 cudaStream_t st) {
    k_sort_triggers<<<1, 1024, 0, st>>>(counter, cap, key_bits, staged, const_cast<uint64_t *>(keys), keys_tmp,
                                        idx_a, idx_b, out, n_out, status);
    return cudaGetLastError();
}

}  // namespace mf
