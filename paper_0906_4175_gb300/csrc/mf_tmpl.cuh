// mf_tmpl.cuh -- 2PN stationary-phase template constants (Sec. 1.1 templates:
// second-order post-Newtonian phase, Newtonian amplitude), usable on host and
// device.  In turns (cycles) and u = f^(-1/3) (f in Hz), with t_c = phi_c = 0:
//   psi(f) = Psi/(2 pi) = -1/8 + c1 u + c2 u^2 + c3 u^3 + c5 u^5,
//   Psi = -pi/4 + 3/(128 eta v^5) [1 + a2 v^2 + a3 v^3 + a4 v^4],  v = (pi M f)^(1/3),
//   a2 = 3715/756 + 55 eta/9,  a3 = -16 pi,
//   a4 = 15293365/508032 + 27145 eta/504 + 3085 eta^2/72,
// since v^-q = (pi M)^(-q/3) u^q.  f_isco = 1/(6^(3/2) pi M); amplitude constant
// A = Mc^(5/6) (any constant cancels in rho).
#pragma once
#include <math.h>

#include "mf_internal.h"

namespace mf {

constexpr double kPiD = 3.14159265358979323846264338327950288;

__host__ __device__ inline void template_constants(double m1, double m2, double *rec) {
    const double M = m1 + m2, Ms = M * kMsunS;
    const double eta = (m1 * m2) / (M * M);
    const double a2 = 3715.0 / 756.0 + 55.0 * eta / 9.0;
    const double a3 = -16.0 * kPiD;
    const double a4 = 15293365.0 / 508032.0 + 27145.0 * eta / 504.0 + 3085.0 * eta * eta / 72.0;
    const double pre = 3.0 / (128.0 * eta) / (2.0 * kPiD);
    const double cb = cbrt(kPiD * Ms);      // (pi M)^(1/3)
    rec[TF_C5] = pre / (cb * cb * cb * cb * cb);
    rec[TF_C3] = pre * a2 / (cb * cb * cb);
    rec[TF_C2] = pre * a3 / (cb * cb);
    rec[TF_C1] = pre * a4 / cb;
    rec[TF_FISCO] = 1.0 / (6.0 * sqrt(6.0) * kPiD * Ms);
    const double Mc = pow(eta, 0.6) * M;
    rec[TF_AMP] = pow(Mc, 5.0 / 6.0);
    rec[TF_M] = M;
    rec[TF_ETA] = eta;
}

// d psi / d m1 and d psi / d m2 as polynomials in u (turns per solar mass):
// d1[i], d2[i] multiply u^p for p = 1, 2, 3, 5.  With c_p = pre a_{5-p}(eta) (pi M)^(-p/3):
//   dc_p/dM = -(p/3) c_p / M,   dc_p/deta = -c_p/eta + pre a'_{5-p}(eta) (pi M)^(-p/3),
//   deta/dm1 = m2 (m2 - m1)/M^3,  deta/dm2 = m1 (m1 - m2)/M^3  (M in solar masses).
__host__ __device__ inline void template_mass_derivs(double m1, double m2, double *d1, double *d2) {
    double rec[kTmplStride];
    template_constants(m1, m2, rec);
    const double M = m1 + m2, Ms = M * kMsunS, eta = rec[TF_ETA];
    const double pre = 3.0 / (128.0 * eta) / (2.0 * kPiD);
    const double cb = cbrt(kPiD * Ms);
    const double c[4] = {rec[TF_C1], rec[TF_C2], rec[TF_C3], rec[TF_C5]};
    const double p[4] = {1.0, 2.0, 3.0, 5.0};
    // pre a'(eta) (pi M)^(-p/3): only p = 3 (a2' = 55/9) and p = 1 (a4' = 27145/504 + 3085 eta/36)
    const double extra[4] = {pre * (27145.0 / 504.0 + 3085.0 * eta / 36.0) / cb, 0.0,
                             pre * (55.0 / 9.0) / (cb * cb * cb), 0.0};
    const double e1 = m2 * (m2 - m1) / (M * M * M);
    const double e2 = m1 * (m1 - m2) / (M * M * M);
    for (int i = 0; i < 4; ++i) {
        const double dM = -(p[i] / 3.0) * c[i] / M;
        const double de = -c[i] / eta + extra[i];
        d1[i] = dM + de * e1;
        d2[i] = dM + de * e2;
    }
}

// Bound on |d^n psi / df^n| (turns / Hz^n) at frequency f: the sum of the
// magnitudes of the n-th derivatives of the four terms c_p u^p, u = f^(-1/3),
//   d^n (f^(-p/3)) / df^n = (-1)^n (p/3)(p/3 + 1)...(p/3 + n - 1) u^(p + 3n).
// Every term decreases with f, so the value at the lowest band frequency
// bounds the whole band.
__host__ __device__ inline double psi_deriv_bound_u(const double *c4, double f, int n) {
    const int pw[4] = {1, 2, 3, 5};
    const double u = 1.0 / cbrt(f);
    double s = 0.0;
    for (int i = 0; i < 4; ++i) {
        const double q = pw[i] / 3.0;
        double fac = 1.0;
        for (int m = 0; m < n; ++m) fac *= (q + m);
        double up = 1.0;
        for (int e = 0; e < pw[i] + 3 * n; ++e) up *= u;
        s += fabs(c4[i]) * fac * up;
    }
    return s;
}

// Anchor spacing D = 2^log2D (bins) for the FP32 quartic Taylor expansion of
// psi about FP64 anchors at the centre of every D bins: the largest D <= 256
// whose fifth-order remainder B5 df^5 (D/2)^5 / 120 stays <= 5e-7 turns and
// whose linear term B1 df D/2 stays <= 16 turns (bounds at the band's lowest
// frequency).
__host__ __device__ inline int anchor_log2D(double B1, double B5, double df) {
    int lg = 0;
    while (lg < 8) {
        const double h = (double)(1 << (lg + 1)) / 2.0;
        const double taylor = B5 * df * df * df * df * df * h * h * h * h * h / 120.0;
        const double mag = B1 * df * h;
        if (taylor > 5e-7 || mag > 16.0) break;
        ++lg;
    }
    return lg;
}

}  // namespace mf
