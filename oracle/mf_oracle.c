/*
 * mf_oracle.c -- plain, slow FP64 CPU oracle for the frequency-domain matched
 * filter of Chung, Wen, Blair, Cannon & Datta, "Application of Graphics
 * Processing Units to Search Pipeline for Gravitational Waves from Coalescing
 * Binaries of Compact Objects" (arXiv:0906.4175), Sec. 1.1, Eqs. (1)-(4).
 * Equations are numbered in order of appearance: (1) z(t), (2) S_n(f),
 * (3) rho(t) = |z|/sigma, (4) sigma^2, (5) chi^2.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  The CUDA path never calls
 * it and shares no code, header, table or constant generator with it.
 *
 * Every routine follows the definitions literally, in FP64, with no blocking,
 * fusion or reordering beyond what the definition states:
 *
 *   s~_k  = dt * sum_n s_n exp(-2 pi i n k / N)                 (data spectrum)
 *   S_k   = Eq. (2) at f_k = k df, f0 = 150 Hz, scale S0         (initial LIGO PSD)
 *   band  = k_lo <= k < k_hi,  k_lo = ceil(f_low/df),
 *           k_hi = min(floor(f_cut/df) + 1, N/2), f_cut = min(f_isco, fs/2)
 *   h~_k  = A f_k^(-7/6) exp(-i Psi(f_k))                        (2PN SPA, Newtonian amplitude, Sec. 1.1)
 *   z_j   = 4 df sum_band h~_k conj(s~_k) / S_k exp(+2 pi i j k / N)   Eq. (1)
 *   sigma^2 = 4 df sum_band |h~_k|^2 / S_k                       Eq. (4)
 *   rho_j = |z_j| / sigma                                        Eq. (3)
 *   chi^2_j = (p / sigma^2) sum_l |z_l,j - z_j / p|^2            Eq. (5), p sub-bands of equal sigma^2 share
 *
 * Readings where the paper is silent (the 2PN phase formula, the ISCO
 * frequency, bin-edge rules, amplitude constant, PSD scale) are stated next to
 * the code that takes them.  The 2PN stationary-phase phase is the standard
 * second-post-Newtonian result of Blanchet, Iyer, Will & Wiseman (1996), the
 * paper's reference for its templates; f_isco = 1/(6^(3/2) pi M) is the
 * test-mass innermost stable circular orbit (the paper's ISCO reference).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846264338327950288
/* G Msun / c^3 in seconds (IAU 2015 nominal solar mass parameter). */
#define OR_MSUN_S 4.925490947e-6

/* ------------------------------------------------------------------------ */
/* FFT: iterative radix-2 Cooley-Tukey, in place, unnormalised.              */
/*   X_k = sum_n x_n exp(sign * 2 pi i n k / n_total)                        */
/* Returns 0, or -1 if n is not a power of two (>= 1).                       */
/* ------------------------------------------------------------------------ */
int or_fft(double *re, double *im, int64_t n, int sign)
{
    if (n < 1 || (n & (n - 1)) != 0) return -1;
    /* bit-reversal permutation */
    for (int64_t i = 1, j = 0; i < n; ++i) {
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    if (n == 1) return 0;
    /* twiddle table w_m = exp(sign 2 pi i m / n), m < n/2 */
    double *wr = (double *)malloc(sizeof(double) * (size_t)(n / 2));
    double *wi = (double *)malloc(sizeof(double) * (size_t)(n / 2));
    if (!wr || !wi) { free(wr); free(wi); return -2; }
    for (int64_t m = 0; m < n / 2; ++m) {
        double a = 2.0 * OR_PI * (double)m / (double)n;
        wr[m] = cos(a);
        wi[m] = (double)sign * sin(a);
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
        int64_t half = len >> 1, step = n / len;
        for (int64_t b = 0; b < n; b += len) {
            for (int64_t j = 0; j < half; ++j) {
                double c = wr[j * step], s = wi[j * step];
                double ur = re[b + j], ui = im[b + j];
                double xr = re[b + j + half], xi = im[b + j + half];
                double vr = xr * c - xi * s, vi = xr * s + xi * c;
                re[b + j] = ur + vr;        im[b + j] = ui + vi;
                re[b + j + half] = ur - vr; im[b + j + half] = ui - vi;
            }
        }
    }
    free(wr); free(wi);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. (2): initial-LIGO one-sided PSD, x = f/f0, times an overall scale S0. */
/* The paper prints no scale; S0 = 1 (whitened units) is the reading, and   */
/* rho does not depend on it.                                               */
/* ------------------------------------------------------------------------ */
double or_psd_eq2(double f, double f0, double S0)
{
    double x = f / f0;
    return S0 * (pow(4.49 * x, -56.0) + 0.16 * pow(x, -4.52) + 0.52 + 0.32 * x * x);
}

/* ------------------------------------------------------------------------ */
/* Template constants for a mass pair (solar masses).                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    double m1, m2;
    double M;      /* total mass, Msun */
    double Ms;     /* total mass, seconds */
    double eta;    /* symmetric mass ratio */
    double Mc;     /* chirp mass, Msun */
    double A;      /* Newtonian amplitude constant: Mc^(5/6) (reading: any constant cancels in rho) */
    double f_isco; /* 1 / (6^(3/2) pi M) */
} or_tmpl;

void or_tmpl_init(double m1, double m2, or_tmpl *t)
{
    t->m1 = m1; t->m2 = m2;
    t->M = m1 + m2;
    t->Ms = (m1 + m2) * OR_MSUN_S;
    t->eta = (m1 * m2) / ((m1 + m2) * (m1 + m2));
    t->Mc = pow(t->eta, 0.6) * t->M;
    t->A = pow(t->Mc, 5.0 / 6.0);
    t->f_isco = 1.0 / (6.0 * sqrt(6.0) * OR_PI * t->Ms);
}

/* 2PN stationary-phase phase, t_c = 0 and phi_c = 0:
 *   Psi(f) = -pi/4 + 3/(128 eta v^5) [1 + (3715/756 + 55 eta/9) v^2 - 16 pi v^3
 *            + (15293365/508032 + 27145 eta/504 + 3085 eta^2/72) v^4],
 *   v = (pi M f)^(1/3), M in seconds.                                         */
double or_psi(double m1, double m2, double f)
{
    or_tmpl t; or_tmpl_init(m1, m2, &t);
    double eta = t.eta;
    double v = cbrt(OR_PI * t.Ms * f);
    double v2 = v * v, v3 = v2 * v, v4 = v2 * v2, v5 = v4 * v;
    double a2 = 3715.0 / 756.0 + 55.0 * eta / 9.0;
    double a3 = -16.0 * OR_PI;
    double a4 = 15293365.0 / 508032.0 + 27145.0 * eta / 504.0 + 3085.0 * eta * eta / 72.0;
    return -OR_PI / 4.0 + 3.0 / (128.0 * eta * v5) * (1.0 + a2 * v2 + a3 * v3 + a4 * v4);
}

/* Band rule of Sec. 1.1: f_low = 40 Hz .. min(Nyquist, f_isco).  Reading:
 * include f = f_low and f <= f_cut, exclude DC and the Nyquist bin.
 *   k_lo = ceil(f_low N / fs),  k_hi = min(floor(f_cut N / fs) + 1, N/2).    */
void or_band(int64_t N, double fs, double f_low, double f_cut,
             int64_t *k_lo, int64_t *k_hi)
{
    double fc = f_cut < 0.5 * fs ? f_cut : 0.5 * fs;
    int64_t lo = (int64_t)ceil(f_low * (double)N / fs);
    int64_t hi = (int64_t)floor(fc * (double)N / fs) + 1;
    if (lo < 1) lo = 1;
    if (hi > N / 2) hi = N / 2;
    if (hi < lo) hi = lo;
    *k_lo = lo; *k_hi = hi;
}

/* h~_k over k = 0..N/2 (zero outside the band).  Returns the band. */
void or_htilde(double m1, double m2, int64_t N, double fs, double f_low,
               double *h_re, double *h_im, int64_t *k_lo, int64_t *k_hi)
{
    or_tmpl t; or_tmpl_init(m1, m2, &t);
    or_band(N, fs, f_low, t.f_isco, k_lo, k_hi);
    double df = fs / (double)N;
    for (int64_t k = 0; k <= N / 2; ++k) { h_re[k] = 0.0; h_im[k] = 0.0; }
    for (int64_t k = *k_lo; k < *k_hi; ++k) {
        double f = (double)k * df;
        double amp = t.A * pow(f, -7.0 / 6.0);
        double psi = or_psi(m1, m2, f);
        h_re[k] = amp * cos(psi);
        h_im[k] = -amp * sin(psi);
    }
}

/* PSD on the bins k = 0..N/2: Eq. (2) (S0 scale) or a caller table. */
void or_psd_bins(int64_t N, double fs, double f0, double S0, double *S)
{
    double df = fs / (double)N;
    S[0] = INFINITY;
    for (int64_t k = 1; k <= N / 2; ++k) S[k] = or_psd_eq2((double)k * df, f0, S0);
}

/* s~_k = dt * DFT(s)_k, k = 0..N/2. */
int or_data_spectrum(const double *s, int64_t N, double fs, double *st_re, double *st_im)
{
    double *re = (double *)malloc(sizeof(double) * (size_t)N);
    double *im = (double *)malloc(sizeof(double) * (size_t)N);
    if (!re || !im) { free(re); free(im); return -2; }
    for (int64_t n = 0; n < N; ++n) { re[n] = s[n]; im[n] = 0.0; }
    int rc = or_fft(re, im, N, -1);
    double dt = 1.0 / fs;
    for (int64_t k = 0; k <= N / 2; ++k) { st_re[k] = dt * re[k]; st_im[k] = dt * im[k]; }
    free(re); free(im);
    return rc;
}

/* Eqs. (1), (3), (4) for one template against one data spectrum.
 * Inputs: s~ and S over k = 0..N/2.  Outputs: z_j (j = 0..N-1), rho_j, sigma. */
int or_filter_template(double m1, double m2, const double *st_re, const double *st_im,
                       const double *S, int64_t N, double fs, double f_low,
                       double *z_re, double *z_im, double *rho, double *sigma_out,
                       int64_t *k_lo_out, int64_t *k_hi_out)
{
    double df = fs / (double)N;
    double *h_re = (double *)malloc(sizeof(double) * (size_t)(N / 2 + 1));
    double *h_im = (double *)malloc(sizeof(double) * (size_t)(N / 2 + 1));
    if (!h_re || !h_im) { free(h_re); free(h_im); return -2; }
    int64_t k_lo, k_hi;
    or_htilde(m1, m2, N, fs, f_low, h_re, h_im, &k_lo, &k_hi);

    /* X_k = h~_k conj(s~_k) / S_k on the band, zero elsewhere (Eq. 1 integrand) */
    for (int64_t k = 0; k < N; ++k) { z_re[k] = 0.0; z_im[k] = 0.0; }
    double sig2 = 0.0;
    for (int64_t k = k_lo; k < k_hi; ++k) {
        double ar = h_re[k], ai = h_im[k];
        double br = st_re[k], bi = -st_im[k];
        z_re[k] = (ar * br - ai * bi) / S[k];
        z_im[k] = (ar * bi + ai * br) / S[k];
        sig2 += (ar * ar + ai * ai) / S[k];             /* Eq. (4) integrand */
    }
    sig2 *= 4.0 * df;
    /* z_j = 4 df sum_k X_k exp(+2 pi i j k / N)   (Eq. 1, Riemann sum) */
    int rc = or_fft(z_re, z_im, N, +1);
    double sigma = sqrt(sig2);
    for (int64_t j = 0; j < N; ++j) {
        z_re[j] *= 4.0 * df; z_im[j] *= 4.0 * df;
        if (rho) rho[j] = sqrt(z_re[j] * z_re[j] + z_im[j] * z_im[j]) / sigma;  /* Eq. (3) */
    }
    if (sigma_out) *sigma_out = sigma;
    if (k_lo_out) *k_lo_out = k_lo;
    if (k_hi_out) *k_hi_out = k_hi;
    free(h_re); free(h_im);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Eq. (5), the chi^2 consistency test of Sec. 1.2: the band integral of     */
/* Eq. (1) is split into p sub-bands that contribute equally to sigma^2, giving */
/* p series z_l(t), and                                                     */
/*   chi^2(t_j) = (p / sigma^2) sum_l |z_l(t_j) - z(t_j)/p|^2.              */
/* Band edges (the paper gives no discretisation): with                     */
/*   c(k) = sum_{k_lo <= k' < k} |h~_k'|^2 / S_k',                          */
/* b_0 = k_lo, b_p = k_hi and, for 0 < l < p, b_l = the smallest k in        */
/* [k_lo, k_hi] with c(k) >= (l/p) c(k_hi).  Sub-band l is b_l <= k < b_{l+1}.*/
/* edges_in (optional, p+1 values) replaces that rule by given edges.        */
/* Outputs: chisq_j and rho_j for j = 0..N-1, edges (p+1), sigma_l^2 (p).    */
/* ------------------------------------------------------------------------ */
int or_chisq_series(double m1, double m2, const double *st_re, const double *st_im,
                    const double *S, int64_t N, double fs, double f_low, int p,
                    const int64_t *edges_in, double *chisq, double *rho,
                    int64_t *edges_out, double *sig2_l_out)
{
    if (p < 1) return -1;
    double df = fs / (double)N;
    int64_t nh = N / 2 + 1;
    double *h_re = (double *)malloc(sizeof(double) * (size_t)nh);
    double *h_im = (double *)malloc(sizeof(double) * (size_t)nh);
    double *c = (double *)malloc(sizeof(double) * (size_t)(nh + 1));
    double *z_re = (double *)malloc(sizeof(double) * (size_t)N);
    double *z_im = (double *)malloc(sizeof(double) * (size_t)N);
    double *zl_re = (double *)malloc(sizeof(double) * (size_t)N);
    double *zl_im = (double *)malloc(sizeof(double) * (size_t)N);
    int64_t *b = (int64_t *)malloc(sizeof(int64_t) * (size_t)(p + 1));
    int rc = 0;
    if (!h_re || !h_im || !c || !z_re || !z_im || !zl_re || !zl_im || !b) { rc = -2; goto done; }
    int64_t k_lo, k_hi;
    or_htilde(m1, m2, N, fs, f_low, h_re, h_im, &k_lo, &k_hi);

    /* cumulative |h|^2/S over the band: c[k - k_lo] = c(k) */
    c[0] = 0.0;
    for (int64_t k = k_lo; k < k_hi; ++k)
        c[k - k_lo + 1] = c[k - k_lo] + (h_re[k] * h_re[k] + h_im[k] * h_im[k]) / S[k];
    double ctot = c[k_hi - k_lo];
    if (edges_in) {
        for (int l = 0; l <= p; ++l) b[l] = edges_in[l];
    } else {
        b[0] = k_lo;
        b[p] = k_hi;
        for (int l = 1; l < p; ++l) {
            double target = ((double)l / (double)p) * ctot;
            int64_t k = k_lo;
            while (k < k_hi && c[k - k_lo] < target) ++k;
            b[l] = k;
        }
    }
    double sig2 = 4.0 * df * ctot;                      /* Eq. (4) */

    /* z over the whole band (Eq. 1) */
    for (int64_t k = 0; k < N; ++k) { z_re[k] = 0.0; z_im[k] = 0.0; }
    for (int64_t k = k_lo; k < k_hi; ++k) {
        double br = st_re[k], bi = -st_im[k];
        z_re[k] = (h_re[k] * br - h_im[k] * bi) / S[k];
        z_im[k] = (h_re[k] * bi + h_im[k] * br) / S[k];
    }
    rc = or_fft(z_re, z_im, N, +1);
    if (rc) goto done;
    for (int64_t j = 0; j < N; ++j) {
        z_re[j] *= 4.0 * df; z_im[j] *= 4.0 * df;
        if (rho) rho[j] = sqrt(z_re[j] * z_re[j] + z_im[j] * z_im[j]) / sqrt(sig2);
        chisq[j] = 0.0;
    }
    /* z_l over each sub-band, and the sum of |z_l - z/p|^2 */
    for (int l = 0; l < p; ++l) {
        double s2 = 0.0;
        for (int64_t k = 0; k < N; ++k) { zl_re[k] = 0.0; zl_im[k] = 0.0; }
        for (int64_t k = b[l]; k < b[l + 1]; ++k) {
            double br = st_re[k], bi = -st_im[k];
            zl_re[k] = (h_re[k] * br - h_im[k] * bi) / S[k];
            zl_im[k] = (h_re[k] * bi + h_im[k] * br) / S[k];
            s2 += (h_re[k] * h_re[k] + h_im[k] * h_im[k]) / S[k];
        }
        if (sig2_l_out) sig2_l_out[l] = 4.0 * df * s2;
        rc = or_fft(zl_re, zl_im, N, +1);
        if (rc) goto done;
        for (int64_t j = 0; j < N; ++j) {
            double dr = 4.0 * df * zl_re[j] - z_re[j] / (double)p;
            double di = 4.0 * df * zl_im[j] - z_im[j] / (double)p;
            chisq[j] += dr * dr + di * di;
        }
    }
    for (int64_t j = 0; j < N; ++j) chisq[j] *= (double)p / sig2;   /* Eq. (5) */
    if (edges_out) for (int l = 0; l <= p; ++l) edges_out[l] = b[l];
done:
    free(h_re); free(h_im); free(c); free(z_re); free(z_im); free(zl_re); free(zl_im); free(b);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Bank filter: per template the peak (argmax of rho, lowest j on ties) and  */
/* every sample with rho_j > thr as a trigger.                               */
/* ------------------------------------------------------------------------ */
typedef struct { double rho; int64_t j; double z_re, z_im; double sigma; int64_t k_lo, k_hi; } or_peak;
typedef struct { int32_t tmpl; int32_t seg; int32_t j; int32_t pad; double rho; double z_re, z_im; } or_trigger;

/* psd: NULL -> Eq. (2) with f0 and S0; else a table over k = 0..N/2.
 * Triggers are written in (template, j) order; *n_trig receives the true
 * count (only the first trig_cap are stored).  Returns the number of threads
 * used, or a negative error. */
int or_filter_bank(const double *m1, const double *m2, int64_t n_t,
                   const double *s, int64_t N, double fs, double f_low,
                   const double *psd, double f0, double S0, double thr, int seg_id,
                   or_peak *peaks, or_trigger *trig, int64_t trig_cap, int64_t *n_trig,
                   int n_threads)
{
    int64_t nh = N / 2 + 1;
    double *st_re = (double *)malloc(sizeof(double) * (size_t)nh);
    double *st_im = (double *)malloc(sizeof(double) * (size_t)nh);
    double *S = (double *)malloc(sizeof(double) * (size_t)nh);
    if (!st_re || !st_im || !S) { free(st_re); free(st_im); free(S); return -2; }
    if (psd) { for (int64_t k = 0; k < nh; ++k) S[k] = psd[k]; }
    else or_psd_bins(N, fs, f0, S0, S);
    if (or_data_spectrum(s, N, fs, st_re, st_im) != 0) { free(st_re); free(st_im); free(S); return -1; }

    /* per-template trigger counts, so that the output order is (template, j) */
    int64_t *cnt = (int64_t *)calloc((size_t)(n_t > 0 ? n_t : 1), sizeof(int64_t));
    int used = 1;
    int err = 0;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#else
    n_threads = 1;
#endif
    /* pass 1: peaks and counts */
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads)
#endif
    {
#ifdef _OPENMP
#pragma omp single
        used = omp_get_num_threads();
#endif
        double *z_re = (double *)malloc(sizeof(double) * (size_t)N);
        double *z_im = (double *)malloc(sizeof(double) * (size_t)N);
        double *rho = (double *)malloc(sizeof(double) * (size_t)N);
        if (!z_re || !z_im || !rho) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            err = -2;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int64_t t = 0; t < n_t; ++t) {
                double sigma; int64_t klo, khi;
                or_filter_template(m1[t], m2[t], st_re, st_im, S, N, fs, f_low,
                                   z_re, z_im, rho, &sigma, &klo, &khi);
                int64_t best = 0;
                int64_t c = 0;
                for (int64_t j = 0; j < N; ++j) {
                    if (rho[j] > rho[best]) best = j;
                    if (rho[j] > thr) ++c;
                }
                peaks[t].rho = rho[best]; peaks[t].j = best;
                peaks[t].z_re = z_re[best]; peaks[t].z_im = z_im[best];
                peaks[t].sigma = sigma; peaks[t].k_lo = klo; peaks[t].k_hi = khi;
                cnt[t] = c;
            }
        }
        free(z_re); free(z_im); free(rho);
    }
    if (err) { free(cnt); free(st_re); free(st_im); free(S); return err; }
    /* exclusive prefix of counts gives each template's first trigger slot */
    int64_t total = 0;
    for (int64_t t = 0; t < n_t; ++t) { int64_t c = cnt[t]; cnt[t] = total; total += c; }
    if (n_trig) *n_trig = total;
    if (trig && trig_cap > 0 && total > 0) {
        /* pass 2: recompute only templates that own stored trigger slots */
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads)
#endif
        {
            double *z_re = (double *)malloc(sizeof(double) * (size_t)N);
            double *z_im = (double *)malloc(sizeof(double) * (size_t)N);
            double *rho = (double *)malloc(sizeof(double) * (size_t)N);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int64_t t = 0; t < n_t; ++t) {
                int64_t first = cnt[t];
                int64_t last = (t + 1 < n_t) ? cnt[t + 1] : total;
                if (first == last || first >= trig_cap || !rho) continue;
                double sigma;
                or_filter_template(m1[t], m2[t], st_re, st_im, S, N, fs, f_low,
                                   z_re, z_im, rho, &sigma, NULL, NULL);
                int64_t o = first;
                for (int64_t j = 0; j < N && o < trig_cap; ++j) {
                    if (rho[j] > thr) {
                        trig[o].tmpl = (int32_t)t; trig[o].seg = seg_id; trig[o].j = (int32_t)j;
                        trig[o].pad = 0; trig[o].rho = rho[j];
                        trig[o].z_re = z_re[j]; trig[o].z_im = z_im[j];
                        ++o;
                    }
                }
            }
            free(z_re); free(z_im); free(rho);
        }
    }
    free(cnt); free(st_re); free(st_im); free(S);
    return used;
}

/* ------------------------------------------------------------------------ */
/* Synthetic data (Sec. 2 test data: stationary coloured Gaussian noise).    */
/* s~_k = sqrt(T S_k / 4) (g1_k + i g2_k) for k_lo <= k < N/2 (reading: the  */
/* data are high-passed at f_low, as every inspiral search conditions its    */
/* input; below f_low Eq. (2) spans ~200 decades), plus frequency-domain     */
/* injections  (snr/sigma) h~_k exp(-2 pi i k j0/N) exp(i phi)  on each      */
/* injection's own band; then s_n = 2 df Re sum_k s~_k exp(+2 pi i n k/N).   */
/* g holds 2*(N/2) normals: g1_k = g[2k], g2_k = g[2k+1].                    */
/* ------------------------------------------------------------------------ */
typedef struct { double m1, m2, snr; int64_t j0; double phi; } or_injection;

int or_synth(const double *g, int64_t N, double fs, double f_low, const double *psd,
             double f0, double S0, const or_injection *inj, int64_t n_inj, double noise_scale,
             double *s_out)
{
    int64_t nh = N / 2 + 1;
    double df = fs / (double)N, T = (double)N / fs;
    double *S = (double *)malloc(sizeof(double) * (size_t)nh);
    double *re = (double *)calloc((size_t)N, sizeof(double));
    double *im = (double *)calloc((size_t)N, sizeof(double));
    double *h_re = (double *)malloc(sizeof(double) * (size_t)nh);
    double *h_im = (double *)malloc(sizeof(double) * (size_t)nh);
    if (!S || !re || !im || !h_re || !h_im) { free(S); free(re); free(im); free(h_re); free(h_im); return -2; }
    if (psd) { for (int64_t k = 0; k < nh; ++k) S[k] = psd[k]; }
    else or_psd_bins(N, fs, f0, S0, S);
    int64_t k_lo = (int64_t)ceil(f_low * (double)N / fs);
    if (k_lo < 1) k_lo = 1;
    for (int64_t k = k_lo; k < N / 2; ++k) {
        double a = noise_scale * sqrt(T * S[k] / 4.0);
        re[k] = a * g[2 * k];
        im[k] = a * g[2 * k + 1];
    }
    for (int64_t i = 0; i < n_inj; ++i) {
        int64_t klo, khi;
        or_htilde(inj[i].m1, inj[i].m2, N, fs, f_low, h_re, h_im, &klo, &khi);
        double sig2 = 0.0;
        for (int64_t k = klo; k < khi; ++k) sig2 += (h_re[k] * h_re[k] + h_im[k] * h_im[k]) / S[k];
        sig2 *= 4.0 * df;
        double amp = inj[i].snr / sqrt(sig2);
        for (int64_t k = klo; k < khi; ++k) {
            /* time shift by j0 samples and constant phase phi */
            double ang = -2.0 * OR_PI * (double)((k * inj[i].j0) % N) / (double)N + inj[i].phi;
            double c = cos(ang), s = sin(ang);
            re[k] += amp * (h_re[k] * c - h_im[k] * s);
            im[k] += amp * (h_re[k] * s + h_im[k] * c);
        }
    }
    int rc = or_fft(re, im, N, +1);
    for (int64_t n = 0; n < N; ++n) s_out[n] = 2.0 * df * re[n];
    free(S); free(re); free(im); free(h_re); free(h_im);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Refinement objective J = rho^2(m1, m2, t) = |z(t)|^2 / sigma^2 with z(t)  */
/* the Eq. (1) sum evaluated directly at continuous t, and its analytic      */
/* gradient d J / d(m1, m2, t).  The band [k_lo, k_hi) is frozen (given).    */
/* h~ = A f^(-7/6) e^(-i Psi):  dh~/dm = h~ (d lnA/dm - i dPsi/dm),          */
/* dz/dt = 4 df sum h~ conj(s~)/S (2 pi i f) e^(2 pi i f t).                  */
/* ------------------------------------------------------------------------ */
static void or_psi_derivs(double m1, double m2, double f, double *psi,
                          double *dpsi_dm1, double *dpsi_dm2)
{
    or_tmpl t; or_tmpl_init(m1, m2, &t);
    double eta = t.eta;
    double v = cbrt(OR_PI * t.Ms * f);
    double a[5], da[5];
    a[0] = 1.0; a[1] = 0.0;
    a[2] = 3715.0 / 756.0 + 55.0 * eta / 9.0;
    a[3] = -16.0 * OR_PI;
    a[4] = 15293365.0 / 508032.0 + 27145.0 * eta / 504.0 + 3085.0 * eta * eta / 72.0;
    da[0] = 0.0; da[1] = 0.0; da[2] = 55.0 / 9.0; da[3] = 0.0;
    da[4] = 27145.0 / 504.0 + 3085.0 * eta / 36.0;
    double sum = 0.0, sum_M = 0.0, sum_eta = 0.0;
    for (int n = 0; n < 5; ++n) {
        double vp = pow(v, (double)(n - 5));
        sum += a[n] * vp;
        sum_M += a[n] * (double)(n - 5) * vp;   /* v d/dv of v^(n-5) */
        sum_eta += da[n] * vp;
    }
    double pre = 3.0 / (128.0 * eta);
    *psi = -OR_PI / 4.0 + pre * sum;
    /* dv/dMs = v / (3 Ms) */
    double dpsi_dMs = pre * sum_M / (3.0 * t.Ms);
    double dpsi_deta = -pre * sum / eta + pre * sum_eta;
    double M = t.M;
    double deta_dm1 = m2 * (m2 - m1) / (M * M * M);
    double deta_dm2 = m1 * (m1 - m2) / (M * M * M);
    *dpsi_dm1 = dpsi_dMs * OR_MSUN_S + dpsi_deta * deta_dm1;
    *dpsi_dm2 = dpsi_dMs * OR_MSUN_S + dpsi_deta * deta_dm2;
}

/* st, S over k = 0..N/2.  Returns J; grad[3] = dJ/d(m1, m2, t). */
double or_refine_objective(double m1, double m2, double tc, const double *st_re, const double *st_im,
                           const double *S, int64_t N, double fs, int64_t k_lo, int64_t k_hi,
                           double *grad)
{
    or_tmpl t; or_tmpl_init(m1, m2, &t);
    double df = fs / (double)N;
    /* d ln A / dm:  A = Mc^(5/6),  ln A = (1/2) ln(m1 m2) - (1/6) ln M */
    double dlnA1 = 0.5 / m1 - 1.0 / (6.0 * t.M);
    double dlnA2 = 0.5 / m2 - 1.0 / (6.0 * t.M);
    double zr = 0, zi = 0, z1r = 0, z1i = 0, z2r = 0, z2i = 0, ztr = 0, zti = 0;
    double sig2 = 0, dsig1 = 0, dsig2 = 0;
    for (int64_t k = k_lo; k < k_hi; ++k) {
        double f = (double)k * df;
        double psi, d1, d2;
        or_psi_derivs(m1, m2, f, &psi, &d1, &d2);
        double amp = t.A * pow(f, -7.0 / 6.0);
        double hr = amp * cos(psi), hi = -amp * sin(psi);
        /* q = h~ conj(s~) / S * exp(2 pi i f t) */
        double br = st_re[k] / S[k], bi = -st_im[k] / S[k];
        double pr = hr * br - hi * bi, pi_ = hr * bi + hi * br;
        double ang = 2.0 * OR_PI * f * tc;
        double c = cos(ang), s = sin(ang);
        double qr = pr * c - pi_ * s, qi = pr * s + pi_ * c;
        zr += qr; zi += qi;
        /* dq/dm = q (dlnA - i dPsi) */
        z1r += dlnA1 * qr + d1 * qi;  z1i += dlnA1 * qi - d1 * qr;
        z2r += dlnA2 * qr + d2 * qi;  z2i += dlnA2 * qi - d2 * qr;
        /* dq/dt = q (2 pi i f) */
        ztr += -2.0 * OR_PI * f * qi;  zti += 2.0 * OR_PI * f * qr;
        double h2 = (hr * hr + hi * hi) / S[k];
        sig2 += h2;
        dsig1 += 2.0 * dlnA1 * h2;
        dsig2 += 2.0 * dlnA2 * h2;
    }
    double w = 4.0 * df;
    zr *= w; zi *= w; z1r *= w; z1i *= w; z2r *= w; z2i *= w; ztr *= w; zti *= w;
    sig2 *= w; dsig1 *= w; dsig2 *= w;
    double z2 = zr * zr + zi * zi;
    double J = z2 / sig2;
    if (grad) {
        double dz2_1 = 2.0 * (zr * z1r + zi * z1i);
        double dz2_2 = 2.0 * (zr * z2r + zi * z2i);
        double dz2_t = 2.0 * (zr * ztr + zi * zti);
        grad[0] = (dz2_1 * sig2 - z2 * dsig1) / (sig2 * sig2);
        grad[1] = (dz2_2 * sig2 - z2 * dsig2) / (sig2 * sig2);
        grad[2] = dz2_t / sig2;
    }
    return J;
}

/* Convenience: J and grad for n triggers theta[i] = (m1, m2, t) on one data
 * segment; the band of each trigger is frozen at its own (m1, m2) unless
 * band[2 i] >= 0, in which case band[2 i], band[2 i + 1] give k_lo, k_hi. */
int or_refine(const double *theta, int64_t n, const double *s, int64_t N, double fs,
              double f_low, const double *psd, double f0, double S0, const int64_t *band,
              double *obj, double *grad)
{
    int64_t nh = N / 2 + 1;
    double *st_re = (double *)malloc(sizeof(double) * (size_t)nh);
    double *st_im = (double *)malloc(sizeof(double) * (size_t)nh);
    double *S = (double *)malloc(sizeof(double) * (size_t)nh);
    if (!st_re || !st_im || !S) { free(st_re); free(st_im); free(S); return -2; }
    if (psd) { for (int64_t k = 0; k < nh; ++k) S[k] = psd[k]; }
    else or_psd_bins(N, fs, f0, S0, S);
    or_data_spectrum(s, N, fs, st_re, st_im);
    for (int64_t i = 0; i < n; ++i) {
        int64_t klo, khi;
        if (band && band[2 * i] >= 0) { klo = band[2 * i]; khi = band[2 * i + 1]; }
        else {
            or_tmpl t; or_tmpl_init(theta[3 * i], theta[3 * i + 1], &t);
            or_band(N, fs, f_low, t.f_isco, &klo, &khi);
        }
        obj[i] = or_refine_objective(theta[3 * i], theta[3 * i + 1], theta[3 * i + 2],
                                     st_re, st_im, S, N, fs, klo, khi, grad ? grad + 3 * i : NULL);
    }
    free(st_re); free(st_im); free(S);
    return 0;
}


/* ------------------------------------------------------------------------ */
/* Trigger clustering (the paper's pipeline reports events, Sec. 3.3; it    */
/* gives no clustering rule).  Reading: single linkage in time with a       */
/* maximum gap of `window` samples, first over the triggers of each          */
/* (template, segment) pair, then over those clusters' loudest members of    */
/* all templates within a segment.  An event is the loudest member (largest */
/* rho; on ties the earlier one in the order of the pass: lower j, then      */
/* lower template).  Input: n triggers sorted by (template, segment, j).     */
/* Output: events sorted by (segment, j) with the number of triggers and of  */
/* per-template clusters merged into each; returns the event count.          */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t tmpl, seg, j, n_trig, n_tmpl, pad; double rho, z_re, z_im; } or_event;

static int or_cmp_seg_j_tmpl(const void *a, const void *b)
{
    const or_event *x = (const or_event *)a, *y = (const or_event *)b;
    if (x->seg != y->seg) return x->seg < y->seg ? -1 : 1;
    if (x->j != y->j) return x->j < y->j ? -1 : 1;
    if (x->tmpl != y->tmpl) return x->tmpl < y->tmpl ? -1 : 1;
    return 0;
}

int64_t or_cluster(const or_trigger *t, int64_t n, int32_t window, or_event *ev, int64_t ev_cap)
{
    or_event *c1 = (or_event *)malloc(sizeof(or_event) * (size_t)(n > 0 ? n : 1));
    if (!c1) return -2;
    int64_t m = 0;
    /* pass 1: per (template, segment), consecutive triggers at most `window` apart */
    for (int64_t i = 0; i < n; ++i) {
        int start = (i == 0) || t[i].tmpl != t[i - 1].tmpl || t[i].seg != t[i - 1].seg ||
                    (int64_t)t[i].j - (int64_t)t[i - 1].j > window;
        if (start) {
            or_event e = {t[i].tmpl, t[i].seg, t[i].j, 1, 1, 0, t[i].rho, t[i].z_re, t[i].z_im};
            c1[m++] = e;
        } else {
            or_event *e = &c1[m - 1];
            e->n_trig += 1;
            if (t[i].rho > e->rho) {
                e->tmpl = t[i].tmpl; e->j = t[i].j; e->rho = t[i].rho; e->z_re = t[i].z_re; e->z_im = t[i].z_im;
            }
        }
    }
    /* pass 2: the clusters' loudest members of all templates, by (segment, j, template) */
    qsort(c1, (size_t)m, sizeof(or_event), or_cmp_seg_j_tmpl);
    int64_t ne = 0;
    or_event cur = {0};
    for (int64_t i = 0; i < m; ++i) {
        int start = (i == 0) || c1[i].seg != c1[i - 1].seg || (int64_t)c1[i].j - (int64_t)c1[i - 1].j > window;
        if (start) {
            if (i > 0) { if (ne < ev_cap) ev[ne] = cur; ++ne; }
            cur = c1[i];
        } else {
            cur.n_trig += c1[i].n_trig;
            cur.n_tmpl += 1;
            if (c1[i].rho > cur.rho) {
                cur.tmpl = c1[i].tmpl; cur.j = c1[i].j; cur.rho = c1[i].rho; cur.z_re = c1[i].z_re; cur.z_im = c1[i].z_im;
            }
        }
    }
    if (m > 0) { if (ne < ev_cap) ev[ne] = cur; ++ne; }
    free(c1);
    return ne;
}
