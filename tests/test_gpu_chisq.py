"""chi^2 consistency test of Eq. (5) (Sec. 1.2) through the C ABI against the
FP64 oracle: every sample of the chi^2 series, the sub-band edges, and the
noise statistic.

Tolerance.  chi^2 = rho_scale^2 (p sum_l |raw_l|^2 - |raw|^2) with
p sum_l |z_l|^2 / sigma^2 = chi^2 + rho^2, so a relative error eps in each z_l
and z moves chi^2 by at most about 2 eps (chi^2 + 2 rho^2).  With eps = 1e-4
(the rho bound of the FP32 path):
  |chi2_gpu - chi2_ref| <= 2e-4 (chi2_ref + 2 rho_ref^2) + 1e-4.
Sub-band edges are integers decided by FP64 comparisons of prefix sums that
the two sides accumulate in different orders (and the CUDA path's per-bin
weights come from FP32 factors), so an edge may sit one bin apart when the
equal-share target falls within rounding of a bin boundary; then the GPU's
edge is checked to satisfy the rule to rounding and the oracle is rerun with
the GPU's edges."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import workloads
from mfgb_testutil import oracle_segment

pytestmark = pytest.mark.gpu


def chi2_tol(ref, rho):
    return 2e-4 * (ref + 2.0 * rho * rho) + 1e-4


@pytest.fixture(scope="module")
def mf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_4175_gb300 import build
    build.build()
    import paper_0906_4175_gb300 as m
    oracle.build()
    return m


def _edge_valid(m1, m2, N, fs, k, l, p, lo, hi):
    """The GPU edge k for sub-band boundary l satisfies the equal-share rule to
    rounding: c(k) >= target and c(k - 1) < target, each up to 1e-9 of c(k_hi)."""
    h, (klo, khi) = oracle.htilde(m1, m2, N, fs, 40.0)
    S = oracle.psd_bins(N, fs)
    q = np.abs(h[klo:khi]) ** 2 / S[klo:khi]
    c = np.concatenate([[0.0], np.cumsum(q)])
    target = l / p * c[-1]
    tol = 1e-9 * c[-1]
    i = k - klo
    return c[i] >= target - tol and (i == 0 or c[i - 1] < target + tol)


def _compare(mf, m1, m2, spec, p=16, f_low=40.0):
    import torch
    s32, s64 = oracle_segment(spec, f_low)
    N, fs = spec.N, spec.fs
    bank = mf.Bank(m1, m2, f_low=f_low)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), fs)
    n = len(m1)
    chi, edges = mf.chisq_series(bank, seg, list(range(n)), p=p)
    chi = chi.cpu().numpy().astype(np.float64)
    edges = edges.cpu().numpy()
    st, S = oracle.data_spectrum(s64, fs), oracle.psd_bins(N, fs)

    def one(t):
        r = oracle.chisq_series(float(m1[t]), float(m2[t]), st, S, N, fs, f_low, p)
        if not np.array_equal(r["edges"], edges[t]):
            d = np.abs(r["edges"] - edges[t])
            assert d.max() <= 1, (t, r["edges"], edges[t])
            for l in np.nonzero(d)[0]:
                assert _edge_valid(float(m1[t]), float(m2[t]), N, fs, int(edges[t][l]), int(l), p,
                                   r["edges"][0], r["edges"][-1]), (t, l)
            r = oracle.chisq_series(float(m1[t]), float(m2[t]), st, S, N, fs, f_low, p, edges=edges[t])
        return r

    with ThreadPoolExecutor(max_workers=16) as ex:
        refs = list(ex.map(one, range(n)))
    worst = 0.0
    for t, r in enumerate(refs):
        err = np.abs(chi[t] - r["chisq"])
        tol = chi2_tol(r["chisq"], r["rho"])
        worst = max(worst, float(np.max(err / tol)))
        assert np.all(err <= tol), (t, float(np.max(err)), int(np.argmax(err / tol)))
    return chi, refs, worst


def test_chisq_tiny_workload_every_sample(mf):
    """16 templates, N = 2^16, one 1.4+1.4 injection at SNR 10: chi^2 at every
    sample and every sub-band edge."""
    wl = workloads.tiny(0)
    _compare(mf, wl.m1, wl.m2, wl.segments[0])


@pytest.mark.parametrize("lg,p", [(10, 16), (12, 4), (14, 16), (17, 16), (18, 7), (19, 5), (21, 8)])
def test_chisq_sizes(mf, lg, p):
    """Every FFT split class (2048-point rows at 2^21; at 2^19 and 2^20 the
    rows kernel over all sub-bands) and several p (including an odd p), heavy
    templates whose band ends far below Nyquist."""
    wl = workloads.small(seed=100 + lg, N=1 << lg, fs=4096.0, n_templates=4, m_lo=1.2, m_hi=12.0)
    _compare(mf, wl.m1, wl.m2, wl.segments[0], p=p)


def test_chisq_bench_segment_sampled(mf):
    """The benchmark's 2^20-sample segment with its 8 injections: chi^2 at
    every sample for the four loudest templates of the bank and two others."""
    import torch
    wl = workloads.scale(0)
    spec = wl.segments[0]
    s32, _ = oracle_segment(spec)
    bank = mf.Bank(wl.m1, wl.m2)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    pk = mf.peaks_to_numpy(mf.filter_bank(bank, [seg], wl.threshold, trig_cap=1 << 20)[0])
    sel = sorted(set([int(x) for x in np.argsort(-pk["rho"])[:4]] + [7, 901]))
    chi, refs, _ = _compare(mf, wl.m1[sel], wl.m2[sel], spec)
    loud = [i for i, t in enumerate(sel) if t in set(int(x) for x in np.argsort(-pk["rho"])[:4])]
    assert all(float(np.max(refs[i]["rho"])) > 7.0 for i in loud)


def test_chisq_two_batches_at_2p20(mf):
    """N = 2^20, p = 16: 34 templates make two batches of the rows kernel (30
    templates' 17 exchanges fill the 4 GiB default budget; the second batch of
    4 runs its one pass-1 launch over all bands in under two waves), every
    sample checked."""
    wl = workloads.small(seed=2020, N=1 << 20, fs=4096.0, n_templates=34, m_lo=1.2, m_hi=6.0)
    _compare(mf, wl.m1, wl.m2, wl.segments[0], p=16)


def test_chisq_rows_timeout_reports_and_recovers(mf):
    """N = 2^19 rows kernel with one list entry's row copies withheld (test
    hook): its waits run out, mf_bank_check reports MF_ETIMEOUT, nothing
    faults, and the next call equals one made before."""
    import torch
    wl = workloads.small(seed=1919, N=1 << 19, fs=4096.0, n_templates=3, m_lo=1.2, m_hi=6.0)
    spec = wl.segments[0]
    s32, _ = oracle_segment(spec)
    bank = mf.Bank(wl.m1, wl.m2)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    a = mf.chisq_series(bank, seg, [0, 1, 2], p=8)[0].cpu().numpy()
    assert bank.check() == 0
    bank.debug_stall(1, spin_limit=2000)
    mf.chisq_series(bank, seg, [0, 1, 2], p=8)
    assert bank.check(allow_timeout=True) == mf._native.MF_ETIMEOUT
    bank.debug_stall(-1)
    b = mf.chisq_series(bank, seg, [0, 1, 2], p=8)[0].cpu().numpy()
    assert bank.check() == 0
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_chisq_noise_mean_and_invalid_index(mf):
    """Pure noise: the mean of chi^2 over all samples of 8 templates is near
    2p - 2; a template index outside the bank gives a zero row."""
    import torch
    N, fs, p = 1 << 18, 4096.0, 16
    spec = workloads.SegmentSpec(N, fs, 4242)
    s32, _ = oracle_segment(spec)
    rng = np.random.default_rng(8)
    m1, m2 = rng.uniform(1.2, 3.0, 8), rng.uniform(1.2, 3.0, 8)
    bank = mf.Bank(m1, m2)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), fs)
    chi, edges = mf.chisq_series(bank, seg, [0, 1, 2, 3, 4, 5, 6, 7, 99, -1], p=p)
    chi = chi.cpu().numpy()
    means = chi[:8].mean(axis=1)
    assert abs(float(means.mean()) - (2 * p - 2)) < 1.5, means
    assert np.all(chi[8:] == 0.0)
    e = edges.cpu().numpy()
    assert np.all(np.diff(e[:8], axis=1) > 0)
