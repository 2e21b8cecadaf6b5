// mf_filter.cuh -- the fused sources and sinks of the bank filter, shared by
// the per-batch kernels (mf_filter.cu) and the persistent scheduler
// (mf_persist.cu).
#pragma once
#include "mf_passes.cuh"

namespace mf {

// ---------------------------------------------------------------------------
// FP64 anchors.  psi(k) = C0 + sum_p c_p u^p, u = (k df)^(-1/3), in turns.  With
// w_p = c_p u^p the k-derivatives are
//   d^n psi/dk^n = (-1)^n sum_p [p (p+3) ... (p+3(n-1)) / 3^n] w_p / k^n,
// so the Taylor coefficients at the anchor centre k_a = g D + D/2 are
//   q1 = -sum p w_p / (3k),  q2 = sum p(p+3) w_p / (18 k^2),
//   q3 = -sum p(p+3)(p+6) w_p / (162 k^3),  q4 = sum p(p+3)(p+6)(p+9) w_p / (1944 k^4).
// psi mod 1 and q1 (which multiplies offsets up to D/2) are formed in FP64 --
// u from an FP32 seed and one FP64 Newton step u <- u (4 - f u^3) / 3 -- and
// q2..q4 in FP32.  Record: float4 (psi mod 1, q1, q2, q3) and float q4.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void anchor_record(double c1, double c2, double c3, double c5, int64_t g, int log2D,
                                              double df, float4 &rec, float &rec4) {
    const int64_t ka = (g << log2D) + ((1 << log2D) >> 1);
    const double f = (double)ka * df;
    double uu = (double)rcbrtf((float)f);
    uu = uu * (4.0 - f * uu * uu * uu) * (1.0 / 3.0);
    const double u2 = uu * uu;
    const double psi = -0.125 + uu * (c1 + uu * (c2 + uu * (c3 + u2 * c5)));
    const double S1 = uu * (c1 + uu * (2.0 * c2 + uu * (3.0 * c3 + u2 * (5.0 * c5))));
    const double ik = df * u2 * uu;   // 1 / k_a
    const double r0 = psi - rint(psi);
    const float uf = (float)uu, ikf = (float)ik;
    const float w1 = (float)c1 * uf, w2 = (float)c2 * uf * uf, w3 = (float)c3 * uf * uf * uf;
    const float w5 = (float)c5 * (uf * uf) * (uf * uf * uf);
    const float S2 = 4.f * w1 + 10.f * w2 + 18.f * w3 + 40.f * w5;
    const float S3 = 28.f * w1 + 80.f * w2 + 162.f * w3 + 440.f * w5;
    const float S4 = 280.f * w1 + 880.f * w2 + 1944.f * w3 + 6160.f * w5;
    const float ik2 = ikf * ikf;
    rec = make_float4((float)r0, (float)(-S1 * ik * (1.0 / 3.0)), S2 * ik2 * (1.f / 18.f),
                      -S3 * ik2 * ikf * (1.f / 162.f));
    rec4 = S4 * ik2 * ik2 * (1.f / 1944.f);
}

// ---------------------------------------------------------------------------
// pass-1 source: X_k = W_k e^{-i Psi_k} on the band, 0 elsewhere; k >= N/2 is
// always outside (one-sided spectrum), so the upper half of every column is 0.
// ---------------------------------------------------------------------------
template <int L, int C, int LG1>
struct TemplateSrc {
    static constexpr bool kHalfZero = true;
    static constexpr bool kSplitTw = true;   // same rounding as the persistent pass 1
    // one anchor record (float4 + float) per non-zero column row, staged per tile
    static constexpr size_t kScratchBytes = (size_t)(L / 2) * (sizeof(float4) + sizeof(float));
    struct Params {
        const float2 *W;
        const UnitInfo *units;
        const float4 *anchors;
        const float *anchors4;
        int anc_stride, log2D;
    };
    const Params &p;
    const int tile, unit, slot;
    float4 *sa;
    float *sa4;
    unsigned *rel = nullptr;   // deferred release (persistent scheduler), done by thread 0 once loads are in flight
    __device__ TemplateSrc(const Params &pp, int tl, int un, int sl, void *scratch)
        : p(pp), tile(tl), unit(un), slot(sl), sa((float4 *)scratch), sa4((float *)((float4 *)scratch + L / 2)) {}
    // All threads of the block call load() (it contains a block barrier).
    __device__ __forceinline__ void load(int seq, int t, float2 *v) const {
        constexpr int T = L / 32;
        const UnitInfo u = p.units[unit];
        const float4 *anc0 = p.anchors + (int64_t)slot * p.anc_stride;   // index: anchor_slot_index(g)
        const float *anc40 = p.anchors4 + (int64_t)slot * p.anc_stride;
        constexpr int LGL = cx_ilog2(L);
        const int k1 = tile * C + seq;
        const int D = 1 << p.log2D;
        float2 w[16];
        bool in[16];
        const int k0 = k1 + (t << LG1);
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int k = k0 + ((r * T) << LG1);
            in[r] = (k >= u.k_lo) && (k < u.k_hi);
            w[r] = in[r] ? __ldg(&p.W[k]) : czero();   // no load outside the band
        }
        if (D >= C && p.log2D <= LG1) {
            // Every column of this tile falls in the same anchor group on a
            // given row n, so the tile needs one anchor per row:
            // g(n) = (tile C >> log2D) + n (N1 >> log2D), record (tile C >> log2D) R + n,
            // staged once in shared memory.
            const int gstep = 1 << (LG1 - p.log2D);
            const int gcol = (tile * C) >> p.log2D;
            const int gbase = gcol - u.g_lo;
            const float4 *acol = anc0 + ((int64_t)gcol << (LGL - 1));
            const float *acol4 = anc40 + ((int64_t)gcol << (LGL - 1));
            for (int n = threadIdx.x; n < L / 2; n += blockDim.x) {
                const int a = gbase + n * gstep;
                if (a >= 0 && a < u.n_anc &&
                    MF_DBG(((int64_t)gcol << (LGL - 1)) + n < p.anc_stride, kDbgAnchor)) {
                    sa[n] = __ldcg(&acol[n]);   // anchors may be rewritten in the same launch (ring)
                    sa4[n] = __ldcg(&acol4[n]);
                }
            }
            release_hook(rel);
            __syncthreads();
            // offset from the anchor centre is the same on every row (D divides N1)
            const float d = (float)((k1 & (D - 1)) - (D >> 1));
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const int n = t + r * T;
                float2 x = czero();
                if (in[r]) {
                    const float4 a = sa[n];
                    const float a4 = sa4[n];
                    float ph = fmaf(fmaf(fmaf(fmaf(a4, d, a.w), d, a.z), d, a.y), d, a.x);
                    ph -= rintf(ph);
                    float sn, cs;
                    __sincosf(6.283185307179586f * ph, &sn, &cs);
                    x = make_float2(fmaf(w[r].x, cs, w[r].y * sn), fmaf(w[r].y, cs, -w[r].x * sn));  // W e^{-i 2 pi ph}
                }
                v[r] = x;
            }
        } else {
            release_hook(rel);
            const int half = D >> 1;
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const int k = k0 + ((r * T) << LG1);
                const int kk = in[r] ? k : u.k_lo;
                const int g = kk >> p.log2D;
                int64_t ai = anchor_slot_index(g, LGL + LG1, LG1, p.log2D);
                if (!MF_DBG(ai >= 0 && ai < p.anc_stride, kDbgAnchor)) ai = 0;
                const float4 a = __ldcg(&anc0[ai]);
                const float a4 = __ldcg(&anc40[ai]);
                const float d = (float)(kk - ((g << p.log2D) + half));
                float ph = fmaf(fmaf(fmaf(fmaf(a4, d, a.w), d, a.z), d, a.y), d, a.x);
                ph -= rintf(ph);
                float sn, cs;
                __sincosf(6.283185307179586f * ph, &sn, &cs);
                const float2 x = make_float2(fmaf(w[r].x, cs, w[r].y * sn), fmaf(w[r].y, cs, -w[r].x * sn));
                v[r] = in[r] ? x : czero();
            }
        }
    }
};

// FP32-only phase (precision-sweep reference): psi evaluated directly in FP32.
template <int L, int C, int LG1>
struct TemplateSrcF32 {
    static constexpr bool kHalfZero = true;
    static constexpr bool kSplitTw = true;
    struct Params {
        const float2 *W;
        const UnitInfo *units;
        const double *tmpl;
        float df;
    };
    static constexpr size_t kScratchBytes = 0;
    const Params &p;
    const int tile, unit;
    __device__ TemplateSrcF32(const Params &pp, int tl, int un, int, void *) : p(pp), tile(tl), unit(un) {}
    __device__ __forceinline__ void load(int seq, int t, float2 *v) const {
        constexpr int T = L / 32;
        const UnitInfo u = p.units[unit];
        const double *Tm = p.tmpl + (int64_t)u.tmpl * kTmplStride;
        const float c1 = (float)Tm[TF_C1], c2 = (float)Tm[TF_C2], c3 = (float)Tm[TF_C3], c5 = (float)Tm[TF_C5];
        const int k1 = tile * C + seq;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int k = k1 + ((t + r * T) << LG1);
            const bool in = (k >= u.k_lo) && (k < u.k_hi);
            const int kk = in ? k : u.k_lo;
            const float2 w = __ldg(&p.W[kk]);
            const float uu = rcbrtf((float)kk * p.df);
            const float u2 = uu * uu;
            float ph = -0.125f + uu * (c1 + uu * (c2 + uu * (c3 + u2 * c5)));
            ph -= rintf(ph);
            float s, c;
            __sincosf(6.283185307179586f * ph, &s, &c);
            const float2 x = make_float2(fmaf(w.x, c, w.y * s), fmaf(w.y, c, -w.x * s));
            v[r] = in ? x : czero();
        }
    }
};

// ---------------------------------------------------------------------------
// pass-2 sink: rho epilogue.  raw_j = row FFT output at j = j2 + N2 j1;
// rho_j = |raw_j| rho_scale.  Tracks the argmax (lowest j on ties) and
// appends every j with |raw_j|^2 > thr2.
// ---------------------------------------------------------------------------
// max(0, a[0], ..., a[R-1]) (NaNs ignored, as by fmaxf) by pairwise halving:
// a dependency chain of log2 R instead of R.
template <int R>
__device__ __forceinline__ float tree_max0(const float *a) {
    if constexpr (R == 1) {
        return fmaxf(0.f, a[0]);
    } else {
        float h[(R + 1) / 2];
#pragma unroll
        for (int i = 0; i < R / 2; ++i) h[i] = fmaxf(a[i], a[i + R / 2]);
        if constexpr (R % 2) h[R / 2] = a[R - 1];
        return tree_max0<(R + 1) / 2>(h);
    }
}

template <int L, int C>
struct RhoSink {
    struct Params {
        const UnitInfo *units;
        float4 *partials;
        mf_trigger *staged;
        uint64_t *keys;
        unsigned long long *counter;
        int64_t cap;
        int log2N2, nblk, seg_idx;
        KeyLayout kl;
    };
    const Params &p;
    const int tile, unit;
    UnitInfo u;
    float bp;
    int bj;
    float2 bz;
    __device__ RhoSink(const Params &pp, int tl, int un, int)
        : p(pp), tile(tl), unit(un), bp(-1.f), bj(0x7fffffff), bz(make_float2(0.f, 0.f)) {
        u = p.units[un];
    }
    template <int R>
    __device__ __forceinline__ void store(int seq, int b, int stride, const float2 *v) {
        const int j2 = tile * C + seq;
        float pw[R];
#pragma unroll
        for (int r = 0; r < R; ++r) pw[r] = fmaf(v[r].x, v[r].x, v[r].y * v[r].y);
        const float m = tree_max0<R>(pw);
        // The butterfly's outputs j2 + N2 (b + r stride) increase with r, so its
        // argmax with the lowest-j tie rule is the first r with pw[r] == m.
        if (m >= bp) {
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
                if (msk == 0u) continue;   // warp-uniform
                const int leader = __ffs(msk) - 1;
                unsigned long long base = 0ull;
                if (lane == leader) base = atomicAdd(p.counter, (unsigned long long)__popc(msk));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (pred) {
                    const unsigned long long slot = base + (unsigned long long)__popc(msk & ((1u << lane) - 1u));
                    if (slot < (unsigned long long)p.cap &&
                        MF_DBG(j2 + ((b + r * stride) << p.log2N2) < (1 << p.kl.j_bits), kDbgOut)) {
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
    // CTA argmax -> partials[unit * nblk + tile]
    __device__ __forceinline__ void finish(float2 *smem) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float op = __shfl_xor_sync(0xffffffffu, bp, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            const float ox = __shfl_xor_sync(0xffffffffu, bz.x, o);
            const float oy = __shfl_xor_sync(0xffffffffu, bz.y, o);
            if (op > bp || (op == bp && oj < bj)) { bp = op; bj = oj; bz = make_float2(ox, oy); }
        }
        __syncthreads();   // the last FFT stage may still be reading shared memory
        float4 *red = reinterpret_cast<float4 *>(smem);
        if (lane == 0) red[warp] = make_float4(bp, __int_as_float(bj), bz.x, bz.y);
        __syncthreads();
        if (threadIdx.x == 0) {
            const int nw = blockDim.x >> 5;
            float4 best = red[0];
            for (int w = 1; w < nw; ++w) {
                const float4 c = red[w];
                const int cj = __float_as_int(c.y), bjj = __float_as_int(best.y);
                if (c.x > best.x || (c.x == best.x && cj < bjj)) best = c;
            }
            p.partials[(int64_t)unit * p.nblk + tile] = best;
        }
    }
};

}  // namespace mf
