"""Shared helpers for the parity tests: run the CUDA path through the C ABI and
the FP64 oracle on the same seeded inputs, and compare.

Tolerances (stated once, used by every GPU test):
  RHO_TOL  err_j = |rho_gpu - rho_ref| / max(rho_ref, 1) <= 1e-4  (FP32 path vs FP64 oracle)
  Peak and trigger indices must agree exactly wherever the decision is not
  within RHO_TOL of a tie or of the threshold.
"""
import numpy as np

import oracle

RHO_TOL = 1e-4

# Refinement (direct Eq. 1 sum at continuous t, FP32 terms and per-thread sums,
# FP64 block totals) against the FP64 oracle:
#   rho^2:     |J_gpu - J_ref| <= REF_OBJ_TOL max(J_ref, 1);
#   gradient:  |g_gpu - g_ref| <= REF_GRAD_RTOL |g_ref| + REF_GRAD_ATOL scale,
#              scale = max over the call's rows of |g_ref| per component.
# Each bin carries a phase error below the anchor remainder bound (5e-7 turns,
# 3e-6 rad) plus FP32 rounding of the Taylor sum and sincos (~1e-6 rad), and
# every FP32 product and partial sum rounds at 6e-8, so a component's error is
# at most a few 1e-6 of the coherent sum of its terms, whose size the largest
# |g| over the rows sets (near a maximum g itself cancels to ~0, hence the
# absolute term).  Measured over N = 2^15 .. 2^20 with both phase forms: rho^2
# error <= 1.3e-6, gradient error <= 7e-7 of the scale and <= 1e-6 of |g| where
# |g| > 0.1 scale; the tolerances are twenty times those.
REF_OBJ_TOL = 3e-5
REF_GRAD_RTOL = 2e-5
REF_GRAD_ATOL = 1.4e-5


def oracle_segment(spec, f_low=40.0):
    """Synthesise the segment with the oracle (FP64) and round it to float32,
    the precision the CUDA path ingests; return (s32, s64_of_s32)."""
    s = oracle.synth(spec.normals(), spec.N, spec.fs, f_low, spec.injections)
    s32 = s.astype(np.float32)
    return s32, s32.astype(np.float64)


def oracle_rho_series(m1, m2, s64, fs, f_low=40.0):
    N = s64.size
    S = oracle.psd_bins(N, fs)
    st = oracle.data_spectrum(s64, fs)
    out = []
    for a, b in zip(m1, m2):
        out.append(oracle.filter_template(float(a), float(b), st, S, N, fs, f_low))
    return out


def gpu_rho_series(mf, bank, seg, n_t, N):
    """Full rho_j for every template via threshold 0 (every sample is a trigger)."""
    peaks, trig, n_trig = mf.filter_bank(bank, [seg], 0.0, trig_cap=n_t * N)
    assert bank.check() == 0
    tr = mf.triggers_to_numpy(trig, n_trig)
    assert tr.size == n_t * N, (tr.size, n_t * N)
    rho = tr["rho"].reshape(n_t, N).astype(np.float64)
    assert np.all(tr["tmpl"].reshape(n_t, N) == np.arange(n_t)[:, None])
    assert np.all(tr["j"].reshape(n_t, N) == np.arange(N)[None, :])
    z = (tr["z_re"] + 1j * tr["z_im"]).reshape(n_t, N)
    return rho, z, mf.peaks_to_numpy(peaks)


def rho_err(gpu, ref):
    return np.abs(gpu - ref) / np.maximum(ref, 1.0)


def peak_index_agrees(rho_ref, j_gpu, j_ref, tol=RHO_TOL):
    """Index must match unless the runner-up (outside +-1 sample of the peak)
    is within 2 tol of the peak."""
    if j_gpu == j_ref:
        return True
    N = rho_ref.size
    r = rho_ref.copy()
    for d in (-1, 0, 1):
        r[(j_ref + d) % N] = -1
    runner = r.max()
    return (rho_ref[j_ref] - runner) / rho_ref[j_ref] <= 2 * tol or (
        abs(rho_ref[j_gpu] - rho_ref[j_ref]) <= 2 * tol * rho_ref[j_ref])


def trigger_sets_agree(gpu_keys, ref_rho, thr, tol=RHO_TOL):
    """gpu_keys: set of (t, j) reported by the GPU; ref_rho: dict t -> oracle
    rho series.  Returns the disagreements that are NOT within tol of thr."""
    ref_keys = set()
    for t, r in ref_rho.items():
        ref_keys.update((t, int(j)) for j in np.nonzero(r > thr)[0])
    bad = []
    for (t, j) in gpu_keys ^ ref_keys:
        r = ref_rho[t][j]
        if abs(r - thr) / thr > tol:
            bad.append((t, j, float(r)))
    return bad
