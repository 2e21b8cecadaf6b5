// mf_chisq.cu -- the chi^2 consistency test of Eq. (5) (Sec. 1.2) as a full
// time series, the computation the paper moved to the GPU: the band of
// Eq. (1) is split into p sub-bands of equal sigma^2 share, each sub-band's
// z_l(t) comes from its own inverse FFT, and
//   chi^2(t) = (p / sigma^2) sum_l |z_l(t) - z(t)/p|^2
//            = rho_scale^2 (p sum_l |raw_l(t)|^2 - |raw(t)|^2)     (sum_l z_l = z),
// with raw the pass-2 output of the filter (rho = |raw| rho_scale).
// Sub-band l is b_l <= k < b_{l+1}: b_0 = k_lo, b_p = k_hi and, for 0 < l < p,
// b_l is the smallest k with P[k] - P[k_lo] >= (l/p)(P[k_hi] - P[k_lo]), P the
// segment's FP64 prefix of f^(-7/3)/S (|h~|^2/S up to the amplitude).
// Each sub-band runs through the filter's own pass 1 (template generation on
// the sub-band only, column IFFTs) and a pass 2 whose sink accumulates
// |raw_l|^2 into the caller's output row; the last, full-band pass 2 turns
// the sum into chi^2.  Neither z_l nor z is stored.
#include "mf_filter.cuh"

namespace mf {

// One block per chi^2 unit: the sub-band edges by binary search in P, then
// p + 1 copies of the unit's full-band UnitInfo (band l = [b_l, b_{l+1}),
// band p = the full band).  A template index outside the bank gives an empty
// band (the output row is zero).
__global__ void k_chisq_units(SegDev seg, const UnitInfo *__restrict__ all, int n_t, const int32_t *__restrict__ tmpl,
                              int n, int p, UnitInfo *__restrict__ out, int64_t *__restrict__ edges) {
    __shared__ int64_t b[kChisqMaxBands + 1];
    const int u = blockIdx.x;
    const int t = tmpl[u];
    UnitInfo full;
    if (t >= 0 && t < n_t) {
        full = all[t];
    } else {   // empty band on template 0's record (keeps every later read in range)
        full = all[0];
        full.k_hi = full.k_lo;
    }
    const int64_t lo = full.k_lo, hi = full.k_hi;
    const double P0 = seg.P[lo], Q = seg.P[hi] - P0;
    for (int l = threadIdx.x; l <= p; l += blockDim.x) {
        int64_t e;
        if (l == 0) {
            e = lo;
        } else if (l == p) {
            e = hi;
        } else {
            const double target = ((double)l / (double)p) * Q;
            int64_t a = lo, c = hi;   // smallest k in [a, c] with P[k] - P0 >= target
            while (a < c) {
                const int64_t m = a + ((c - a) >> 1);
                if (seg.P[m] - P0 >= target) c = m;
                else a = m + 1;
            }
            e = a;
        }
        b[l] = e;
        if (edges) edges[(int64_t)u * (p + 1) + l] = e;
    }
    __syncthreads();
    for (int l = threadIdx.x; l <= p; l += blockDim.x) {
        UnitInfo x = full;
        if (l < p) {
            x.k_lo = (int32_t)b[l];
            x.k_hi = (int32_t)b[l + 1];
        }
        out[(int64_t)l * n + u] = x;
    }
}

// pass-2 sinks.  The CTA owns rows j2 = tile C .. tile C + C - 1, i.e. C
// consecutive samples out of every N2, so per-element global accesses from
// the butterflies would touch one 32-byte sector per lane.  Each thread
// therefore parks |raw|^2 of its outputs in its sequence's shared-memory row
// (free once every thread of the sequence has read its last stage: the warp
// for rows of up to 1024 points, the CTA for 2048), and finish() moves the
// C x N1 tile to the unit's output row with the C consecutive samples of each
// j1 on consecutive threads.
template <int L, int C>
__device__ __forceinline__ float *chi_tile_row(int seq) {
    extern __shared__ float2 chi_smem[];
    return reinterpret_cast<float *>(chi_smem + seq * SeqStride<L, C>::value);
}

template <int L, int C>
__device__ __forceinline__ void chi_park(int seq, int b, int stride, const float2 *v, int R) {
    float *row = chi_tile_row<L, C>(seq);
    if constexpr (L / 32 <= 32) __syncwarp();   // the sequence's threads have read their last-stage inputs
    else __syncthreads();                        // (a 2048-point sequence spans two warps; every thread gets here once)
#pragma unroll 32
    for (int r = 0; r < R; ++r) row[b + r * stride] = fmaf(v[r].x, v[r].x, v[r].y * v[r].y);
}

// mode 0: acc = |raw|^2, 1: acc += |raw|^2, 2: acc = rs2 (p acc - |raw|^2).
// Rows of up to 2048 points go through the shared-memory tile; longer rows
// would update the output element by element from the butterflies.
template <int L, int C>
struct ChiSink {
    static constexpr bool kTile = (L / 32) <= 64;
    struct Params { float *acc; const UnitInfo *units; int log2N2, log2N, mode; float pf; };
    const Params &p;
    const int tile, unit;
    float rs2;
    __device__ ChiSink(const Params &pp, int tl, int un, int) : p(pp), tile(tl), unit(un), rs2(0.f) {
        if (p.mode == 2) {
            const float rs = p.units[un].rho_scale;
            rs2 = rs * rs;
        }
    }
    __device__ __forceinline__ void update(float *q, float pw) const {
        if (p.mode == 0) *q = pw;
        else if (p.mode == 1) *q += pw;
        else *q = rs2 * fmaf(p.pf, *q, -pw);
    }
    template <int R>
    __device__ __forceinline__ void store(int seq, int b, int stride, const float2 *v) const {
        if constexpr (kTile) {
            chi_park<L, C>(seq, b, stride, v, R);
        } else {
            float *a = p.acc + ((int64_t)unit << p.log2N) + tile * C + seq;
#pragma unroll
            for (int r = 0; r < R; ++r)
                update(a + ((int64_t)(b + r * stride) << p.log2N2), fmaf(v[r].x, v[r].x, v[r].y * v[r].y));
        }
    }
    __device__ __forceinline__ void finish(float2 *) const {
        if constexpr (kTile) {
            __syncthreads();
            float *a = p.acc + ((int64_t)unit << p.log2N) + tile * C;
            // C L elements over C (L / 32) threads: 32 per thread, issued in
            // groups of 8 loads before their read-modify-writes
            constexpr int NT = C * (L / 32);
            constexpr int G = 8;
            static_assert((C * L) % (NT * G) == 0, "tile split");
#pragma unroll 1
            for (int base = 0; base < C * L; base += NT * G) {
                float pw[G], old[G];
                float *q[G];
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int idx = base + g * NT + (int)threadIdx.x;
                    const int seq = idx % C, j1 = idx / C;
                    q[g] = a + seq + ((int64_t)j1 << p.log2N2);
                    pw[g] = chi_tile_row<L, C>(seq)[j1];
                    old[g] = p.mode == 0 ? 0.f : __ldcg(q[g]);
                }
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const float x = p.mode == 0 ? pw[g] : (p.mode == 1 ? old[g] + pw[g] : rs2 * fmaf(p.pf, old[g], -pw[g]));
                    __stcg(q[g], x);
                }
            }
        }
    }
};

namespace {
struct ChiPass2Op {
    const SegDev &seg;
    const UnitInfo *units;
    int unit0, n_units;
    const float2 *exch;
    float *acc;
    int mode;   // 0: first sub-band (store), 1: later sub-band (add), 2: full band (chi^2)
    int p;
    cudaStream_t st;
    template <int N2, int N1>
    cudaError_t run() {
        constexpr int C = seqs_per_cta<N1>(N2);
        const dim3 grid(N2 / C, n_units);
        typename RowSrc<N1, C>::Params sp{exch, seg.log2N1, seg.log2N};
        typename ChiSink<N1, C>::Params kp{acc, units, seg.log2N2, seg.log2N, mode, (float)p};
        return run_pass<N1, C, false, +1, RowSrc<N1, C>, ChiSink<N1, C>>(grid, sp, kp, st, unit0);
    }
};

struct ChiAttrOp {
    template <int N2, int N1>
    cudaError_t run() {
        constexpr int C = seqs_per_cta<N1>(N2);
        return set_pass_attrs<N1, C, false, +1, RowSrc<N1, C>, ChiSink<N1, C>>();
    }
};
}  // namespace

cudaError_t launch_chisq_units(const SegDev &seg, const UnitInfo *all, int n_t, const int32_t *tmpl, int n, int p,
                               UnitInfo *out, int64_t *edges, cudaStream_t st) {
    if (p < 1 || p > kChisqMaxBands) return cudaErrorInvalidValue;
    k_chisq_units<<<n, 128, 0, st>>>(seg, all, n_t, tmpl, n, p, out, edges);
    return cudaGetLastError();
}

cudaError_t launch_chisq_pass2(const SegDev &seg, const UnitInfo *units, int unit0, int n_units, const float2 *exch,
                               float *acc, int mode, int p, cudaStream_t st) {
    ChiPass2Op op{seg, units, unit0, n_units, exch, acc, mode, p, st};
    return dispatch_split(seg.log2N, op);
}

cudaError_t chisq_kernel_attributes() {
    {
        cudaError_t e0 = init_twiddle_tables();
        if (e0 != cudaSuccess) return e0;
    }
    for (int lg = 10; lg <= 22; ++lg) {
        ChiAttrOp op;
        cudaError_t e = dispatch_split(lg, op);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace mf
