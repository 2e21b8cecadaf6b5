"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs: Eqs. (1), (3), (4) of arXiv:0906.4175 with the Sec. 1.1 templates.

Every comparison uses RHO_TOL = 1e-4 on err_j = |rho_gpu - rho_ref| / max(rho_ref, 1).
"""
import os

import numpy as np
import pytest

import oracle
import workloads
from mfgb_testutil import (REF_GRAD_ATOL, REF_GRAD_RTOL, REF_OBJ_TOL, RHO_TOL, gpu_rho_series, oracle_rho_series,
                           oracle_segment, peak_index_agrees, rho_err, trigger_sets_agree)

pytestmark = pytest.mark.gpu


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


def _full_compare(mf, m1, m2, spec, f_low=40.0, phase_mode=0, tol=RHO_TOL):
    s32, s64 = oracle_segment(spec, f_low)
    import torch
    bank = mf.Bank(m1, m2, f_low=f_low, phase_mode=phase_mode)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    rho_g, z_g, peaks = gpu_rho_series(mf, bank, seg, len(m1), spec.N)
    ref = oracle_rho_series(m1, m2, s64, spec.fs, f_low)
    worst = 0.0
    for t, r in enumerate(ref):
        e = rho_err(rho_g[t], r["rho"])
        worst = max(worst, float(e.max()))
        jr = int(np.argmax(r["rho"]))
        assert peak_index_agrees(r["rho"], int(peaks["j"][t]), jr), (t, peaks["j"][t], jr)
        assert abs(peaks["rho"][t] - r["rho"][jr]) / max(r["rho"][jr], 1) <= tol
        # z itself (Eq. 1, amplitude A = Mc^(5/6)): relative to sigma
        ez = np.abs(z_g[t] - r["z"]) / r["sigma"]
        assert ez.max() <= tol, (t, ez.max())
    assert worst <= tol, worst
    return worst


def test_tiny_workload_full_series(mf):
    """16 templates, N = 2^16, fs = 2048, one injection: every rho_j."""
    wl = workloads.tiny(0)
    _full_compare(mf, wl.m1, wl.m2, wl.segments[0])


@pytest.mark.parametrize("lg,fs", [(10, 4096.0), (11, 4096.0), (12, 4096.0), (13, 2048.0), (14, 4096.0),
                                   (15, 4096.0), (17, 4096.0), (18, 4096.0), (19, 4096.0), (20, 4096.0)])
def test_sizes_full_series(mf, lg, fs):
    """Every supported FFT split from 32x32 up to 512x512 (ragged tails: the
    heaviest templates cut at f_isco far below Nyquist)."""
    N = 1 << lg
    wl = workloads.small(seed=lg, N=N, fs=fs, n_templates=5, m_lo=1.2, m_hi=12.0)
    _full_compare(mf, wl.m1, wl.m2, wl.segments[0])


@pytest.mark.parametrize("lg", [18, 19, 20, 21, 22])
def test_alternative_split_full_series(mf, monkeypatch, lg):
    """The autotuner's alternative four-step split of N (2^18: 256 x 1024,
    2^19: 1024 x 512, 2^20: 512 x 2048, 2^21: 2048 x 1024, 2^22: 1024 x 4096
    columns x rows) through every kernel form of the per-batch schedule:
    every rho_j and z against the oracle."""
    monkeypatch.setenv("MFGB_SCHED", "batch")
    monkeypatch.setenv("MFGB_SPLIT_ALT", "1")
    wl = workloads.small(seed=100 + lg, N=1 << lg, fs=4096.0, n_templates=2 if lg >= 20 else 3,
                         m_lo=1.2, m_hi=9.0)
    _full_compare(mf, wl.m1, wl.m2, wl.segments[0])
    if lg <= 19:
        monkeypatch.setenv("MFGB_P1PF", "0")   # per-tile pass 1 on the same split
        monkeypatch.setenv("MFGB_P2ROWS", "0")
        _full_compare(mf, wl.m1, wl.m2, wl.segments[0])


def test_largest_segments_sampled(mf):
    """N = 2^21 and 2^22 (1024x2048, 2048x2048 splits), two templates each."""
    import torch
    for lg in (21, 22):
        N = 1 << lg
        wl = workloads.small(seed=lg, N=N, fs=4096.0, n_templates=2, m_lo=1.5, m_hi=8.0)
        spec = wl.segments[0]
        s32, s64 = oracle_segment(spec)
        bank = mf.Bank(wl.m1, wl.m2)
        seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
        peaks, trig, n = mf.filter_bank(bank, [seg], 5.0, trig_cap=1 << 16)
        assert bank.check() == 0
        pk = mf.peaks_to_numpy(peaks)
        ref = oracle_rho_series(wl.m1, wl.m2, s64, spec.fs)
        tr = mf.triggers_to_numpy(trig, n)
        for t, r in enumerate(ref):
            jr = int(np.argmax(r["rho"]))
            assert peak_index_agrees(r["rho"], int(pk["j"][t]), jr)
            assert abs(pk["rho"][t] - r["rho"][jr]) / max(1, r["rho"][jr]) <= RHO_TOL
        gk = {(int(a), int(b)) for a, b in zip(tr["tmpl"], tr["j"])}
        assert trigger_sets_agree(gk, {t: r["rho"] for t, r in enumerate(ref)}, 5.0) == []
        for x in tr:
            assert abs(x["rho"] - ref[x["tmpl"]]["rho"][x["j"]]) / max(1, x["rho"]) <= RHO_TOL


def test_phase_fp64_mode_matches(mf):
    wl = workloads.small(seed=3, N=1 << 14, fs=4096.0, n_templates=4)
    _full_compare(mf, wl.m1, wl.m2, wl.segments[0], phase_mode=mf.MF_PHASE_FP64)


def test_scale_workload_sampled(mf):
    """The benchmark's workload (1024 templates, N = 2^20, 8 injections, thr 6)
    in the benchmark's launch configuration; peaks and triggers of a sample of
    templates (those nearest the injections plus random ones) against the oracle."""
    import torch
    wl = workloads.scale(0)
    spec = wl.segments[0]
    s32, s64 = oracle_segment(spec)
    bank = mf.Bank(wl.m1, wl.m2)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    peaks, trig, n = mf.filter_bank(bank, [seg], wl.threshold, trig_cap=1 << 22)
    assert bank.check() == 0
    pk = mf.peaks_to_numpy(peaks)
    tr = mf.triggers_to_numpy(trig, n)
    assert tr.size == int(n.item())
    # sorted by (tmpl, j)
    key = tr["tmpl"].astype(np.int64) * spec.N + tr["j"]
    assert np.all(np.diff(key) > 0)
    # sample: the loudest template per injection, plus 6 random templates
    rng = np.random.default_rng(0)
    loud = list(np.argsort(-pk["rho"])[:4])
    sample = sorted(set(int(x) for x in loud + list(rng.choice(wl.n_templates, 6, replace=False))))
    ref = oracle_rho_series(wl.m1[sample], wl.m2[sample], s64, spec.fs)
    ref_by_t = {}
    for t, r in zip(sample, ref):
        jr = int(np.argmax(r["rho"]))
        assert peak_index_agrees(r["rho"], int(pk["j"][t]), jr), (t, pk["j"][t], jr)
        assert abs(pk["rho"][t] - r["rho"][jr]) / max(1, r["rho"][jr]) <= RHO_TOL
        ref_by_t[t] = r["rho"]
    gk = {(int(a), int(b)) for a, b in zip(tr["tmpl"], tr["j"]) if int(a) in ref_by_t}
    assert trigger_sets_agree(gk, ref_by_t, wl.threshold) == []
    for x in tr:
        if int(x["tmpl"]) in ref_by_t:
            r = ref_by_t[int(x["tmpl"])][x["j"]]
            assert abs(x["rho"] - r) / max(1, r) <= RHO_TOL
    # injections at lattice masses are recovered near their SNR
    assert pk["rho"].max() > 8.0


def test_synth_matches_oracle(mf):
    for N, fs, n_inj in [(1 << 12, 4096.0, 1), (1 << 16, 2048.0, 3), (1 << 20, 4096.0, 8)]:
        wl = workloads.small(seed=N, N=N, fs=fs, n_templates=1, n_inj=n_inj)
        spec = wl.segments[0]
        g = spec.normals()
        ref = oracle.synth(g, N, fs, 40.0, spec.injections)
        got = mf.synth_segment(g, N, fs, 40.0, spec.injections).cpu().numpy().astype(np.float64)
        err = np.abs(got - ref).max() / np.sqrt(np.mean(ref ** 2))
        assert err < 2e-5, (N, err)


def test_determinism_and_order_independence(mf):
    import torch
    wl = workloads.small(seed=5, N=1 << 15, fs=4096.0, n_templates=12)
    spec = wl.segments[0]
    s32, _ = oracle_segment(spec)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    bank = mf.Bank(wl.m1, wl.m2)
    a = [x.cpu().numpy().copy() for x in mf.filter_bank(bank, [seg], 4.0, trig_cap=1 << 18)]
    b = [x.cpu().numpy().copy() for x in mf.filter_bank(bank, [seg], 4.0, trig_cap=1 << 18)]
    for x, y in zip(a, b):
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8))
    perm = np.random.default_rng(1).permutation(12)
    bank2 = mf.Bank(wl.m1[perm], wl.m2[perm])
    p2, t2, n2 = mf.filter_bank(bank2, [seg], 4.0, trig_cap=1 << 18)
    pa = a[0].view(mf.PEAK_DTYPE).reshape(-1)
    pb = mf.peaks_to_numpy(p2)
    assert np.array_equal(pa[perm].view(np.uint8), pb.view(np.uint8))
    assert int(n2.item()) == int(a[2][0])


def test_mirror_masses_identical(mf):
    import torch
    spec = workloads.small(seed=9, N=1 << 14).segments[0]
    s32, _ = oracle_segment(spec)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    bank = mf.Bank([1.3, 2.7], [2.7, 1.3])
    p, _, _ = mf.filter_bank(bank, [seg], 100.0, trig_cap=0)
    pk = mf.peaks_to_numpy(p)
    assert pk[0].tobytes() == pk[1].tobytes()


def test_overflow_keeps_true_count(mf):
    import torch
    spec = workloads.small(seed=2, N=1 << 13).segments[0]
    s32, _ = oracle_segment(spec)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    bank = mf.Bank([1.4, 2.0, 3.0], [1.4, 1.5, 2.5])
    _, _, n_full = mf.filter_bank(bank, [seg], 1.0, trig_cap=1 << 16)
    assert bank.check() == 0
    total = int(n_full.item())
    assert total > 100
    _, trig, n = mf.filter_bank(bank, [seg], 1.0, trig_cap=37)
    assert bank.check() == mf._native.MF_EOVERFLOW
    assert int(n.item()) == total
    tr = mf.triggers_to_numpy(trig, n)
    assert tr.size == 37
    key = tr["tmpl"].astype(np.int64) * spec.N + tr["j"]
    assert np.all(np.diff(key) > 0)
    assert np.all(tr["rho"] > 1.0)
    # nothing above an enormous threshold
    _, _, n0 = mf.filter_bank(bank, [seg], 1e6, trig_cap=8)
    assert bank.check() == 0 and int(n0.item()) == 0


def test_multi_segment_call_equals_separate_calls(mf):
    import torch
    specs = [workloads.small(seed=s, N=N, fs=4096.0).segments[0] for s, N in ((1, 1 << 12), (2, 1 << 14))]
    segs = [mf.Segment(torch.from_numpy(oracle_segment(sp)[0]).cuda(), sp.fs) for sp in specs]
    m1 = np.array([1.3, 1.9, 2.4, 3.3, 1.1])
    m2 = np.array([1.2, 1.7, 2.4, 1.5, 1.0])
    bank = mf.Bank(m1, m2)
    p, t, n = mf.filter_bank(bank, segs, 3.5, trig_cap=1 << 16)
    pk = mf.peaks_to_numpy(p).reshape(5, 2)
    tr = mf.triggers_to_numpy(t, n)
    for si, sg in enumerate(segs):
        p1, t1, n1 = mf.filter_bank(bank, [sg], 3.5, trig_cap=1 << 16)
        assert np.array_equal(mf.peaks_to_numpy(p1).view(np.uint8), pk[:, si].copy().view(np.uint8))
        t1 = mf.triggers_to_numpy(t1, n1)
        sub = tr[tr["seg"] == si]
        assert np.array_equal(sub[["tmpl", "j", "rho", "z_re", "z_im"]], t1[["tmpl", "j", "rho", "z_re", "z_im"]])


@pytest.mark.parametrize("f_low", [30.0, 60.0])
def test_mixed_rates_and_f_low_one_call(mf, f_low):
    """Segments of three sample rates (1024, 2048, 4096 Hz) and lengths in ONE
    call, with a lower cut-off other than 40 Hz (the band rule of Sec. 1.1:
    k_lo = ceil(f_low N / fs), f_cut = min(f_isco, fs/2), so the heavier
    templates end below Nyquist at 4096 Hz and the lighter ones are cut at
    Nyquist at 1024 Hz): every rho_j and z_j of every (template, segment)
    against the oracle run at that f_low.  (Data with content below f_low:
    test_data_content_far_below_f_low.)"""
    import torch
    m1 = np.array([1.25, 1.6, 2.9, 4.8, 9.0, 1.4])
    m2 = np.array([1.2, 1.45, 2.1, 3.5, 7.5, 1.4])
    specs = [workloads.small(seed=40 + i, N=N, fs=fs, n_templates=1, m_lo=1.2, m_hi=3.0).segments[0]
             for i, (N, fs) in enumerate(((1 << 13, 1024.0), (1 << 15, 2048.0), (1 << 17, 4096.0)))]
    data = [oracle_segment(sp, f_low) for sp in specs]
    segs = [mf.Segment(torch.from_numpy(s32).cuda(), sp.fs) for (s32, _), sp in zip(data, specs)]
    bank = mf.Bank(m1, m2, f_low=f_low)
    n_t, n_seg = len(m1), len(segs)
    total = n_t * sum(sp.N for sp in specs)
    p, t, n = mf.filter_bank(bank, segs, 0.0, trig_cap=total)
    assert bank.check() == 0
    tr = mf.triggers_to_numpy(t, n)
    assert tr.size == total
    pk = mf.peaks_to_numpy(p).reshape(n_t, n_seg)
    for si, (sp, (_, s64)) in enumerate(zip(specs, data)):
        ref = oracle_rho_series(m1, m2, s64, sp.fs, f_low)
        for ti, r in enumerate(ref):
            sel = tr[(tr["tmpl"] == ti) & (tr["seg"] == si)]
            assert sel.size == sp.N and np.array_equal(sel["j"], np.arange(sp.N))
            e = rho_err(sel["rho"].astype(np.float64), r["rho"])
            assert e.max() <= RHO_TOL, (si, ti, float(e.max()))
            ez = np.abs(sel["z_re"] + 1j * sel["z_im"] - r["z"]) / r["sigma"]
            assert ez.max() <= RHO_TOL, (si, ti, float(ez.max()))
            jr = int(np.argmax(r["rho"]))
            assert peak_index_agrees(r["rho"], int(pk[ti, si]["j"]), jr), (si, ti)


@pytest.mark.parametrize("f_noise,N,fs", [(20.0, 1 << 16, 4096.0), (15.0, 1 << 17, 2048.0)])
def test_data_content_far_below_f_low(mf, f_noise, N, fs):
    """Eq. (2)-coloured noise from f_noise = 15-20 Hz, below the filter's
    f_low = 40 Hz: the seismic wall of Eq. (2) makes that content 10^5 - 10^8
    times the in-band amplitude, yet every rho_j and z_j stays within the FP32
    path's bound of the oracle (run on the same float32 samples) because the
    segment's forward FFT runs in FP64.  The FP32 forward FFT (MF_COND_FP32
    refresh) on the same samples misses the bound by orders of magnitude."""
    import torch
    m1 = np.array([1.3, 2.2, 5.0])
    m2 = np.array([1.25, 1.9, 3.0])
    inj = np.zeros(1, dtype=oracle.INJ_DTYPE)
    inj[0] = (2.2, 1.9, 12.0, N // 3, 0.4)
    spec = workloads.SegmentSpec(N, fs, int(f_noise) * 7 + 3, inj)
    s32 = oracle.synth(spec.normals(), N, fs, f_noise, spec.injections).astype(np.float32)
    s64 = s32.astype(np.float64)
    bank = mf.Bank(m1, m2)
    s_dev = torch.from_numpy(s32).cuda()
    seg = mf.Segment(s_dev, fs)
    rho_g, z_g, pk = gpu_rho_series(mf, bank, seg, len(m1), N)
    ref = oracle_rho_series(m1, m2, s64, fs, 40.0)
    errs = []
    for t, r in enumerate(ref):
        e = rho_err(rho_g[t], r["rho"])
        assert e.max() <= RHO_TOL, (t, float(e.max()))
        assert (np.abs(z_g[t] - r["z"]) / r["sigma"]).max() <= RHO_TOL
        assert peak_index_agrees(r["rho"], int(pk["j"][t]), int(np.argmax(r["rho"])))
        errs.append(float(e.max()))
    seg.set_conditioning("fp32")
    seg.refresh(s_dev)
    rho_32, _, _ = gpu_rho_series(mf, bank, seg, len(m1), N)
    e32 = max(float(rho_err(rho_32[t], r["rho"]).max()) for t, r in enumerate(ref))
    assert e32 > 10 * RHO_TOL and e32 > 100 * max(errs), (e32, errs)


@pytest.mark.parametrize("lg", [12, 20])
def test_degenerate_bands(mf, lg):
    """Templates whose ISCO cut leaves 1, 2 and 3 bins above f_low (mid-bin
    f_isco, so the integer band is not a rounding decision), beside an
    ordinary one: the full rho and z series against the oracle (a 1-bin band
    gives a rho series that is flat up to rounding, so the peak index is a
    tie).  At 2^20 the staged pass 1 and the rows kernel run them.  A
    template cut below f_low is refused."""
    import torch
    N, fs = 1 << lg, 4096.0
    c = oracle.f_isco(1.0, 1.0) * 2.0           # f_isco(m, m) = c / (2 m)
    ms = [c / (2.0 * (40.0 + (nb - 0.5) * fs / N)) for nb in (1, 2, 3)]
    for nb, m in zip((1, 2, 3), ms):
        lo, hi = oracle.band(N, fs, 40.0, min(oracle.f_isco(m, m), fs / 2))
        assert hi - lo == nb
    m1 = np.array(ms + [1.4])
    spec = workloads.small(seed=70 + lg, N=N, fs=fs).segments[0]
    _full_compare(mf, m1, m1.copy(), spec)
    bank = mf.Bank([c / (2.0 * 39.0)], [c / (2.0 * 39.0)])
    seg = mf.Segment(torch.zeros(N, device="cuda"), fs)
    with pytest.raises(mf.MFError) as ei:
        mf.filter_bank(bank, [seg], 6.0)
    assert "MF_EINVAL" in str(ei.value)


@pytest.mark.parametrize("snr", [200.0, 2000.0])
def test_loud_injection_envelope(mf, snr):
    """FP32 round-off in the transforms scales with the loudest signal of the
    segment, so the error at noise-level samples grows linearly with the
    injection's SNR: within RHO_TOL up to SNR ~ 1000 (the paper's workloads
    use SNR 8-20), RHO_TOL * SNR / 1000 beyond.  One 1.4+1.4 injection, N = 2^16,
    the full series of the matched and a mismatched template."""
    import torch
    N, fs = 1 << 16, 4096.0
    inj = np.zeros(1, dtype=oracle.INJ_DTYPE)
    inj[0] = (1.4, 1.4, snr, 12345, 0.7)
    spec = workloads.SegmentSpec(N, fs, 91, inj)
    s32, s64 = oracle_segment(spec)
    m1, m2 = np.array([1.4, 1.6]), np.array([1.4, 1.3])
    bank = mf.Bank(m1, m2)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), fs)
    rho_g, _, pk = gpu_rho_series(mf, bank, seg, 2, N)
    ref = oracle_rho_series(m1, m2, s64, fs)
    bound = RHO_TOL * max(1.0, snr / 1000.0)
    for t in range(2):
        assert rho_err(rho_g[t], ref[t]["rho"]).max() <= bound, t
    assert abs(ref[0]["rho"].max() / snr - 1) < 0.05 and int(pk["j"][0]) == (N - 12345) % N


def test_stage_profile_counts(mf, monkeypatch):
    """mf_bank_profile: per-stage launches match the batches (two of 24 and
    one of 16 templates), the algorithmic bytes are exact (pass 2 reads
    8 N per template; pass 1 writes 8 N and reads the 8 K_t-byte W band,
    K_t from the oracle's band rule, plus the anchor records the anchor stage
    reports), a read clears the counters, and results with profiling on
    equal those without."""
    import torch
    monkeypatch.setenv("MFGB_SCHED", "batch")
    monkeypatch.setenv("MFGB_BATCH", "24")
    wl = workloads.small(seed=9, N=1 << 17, fs=4096.0, n_templates=64)
    spec = wl.segments[0]
    s32, _ = oracle_segment(spec)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    bank = mf.Bank(wl.m1, wl.m2)
    ref = mf.peaks_to_numpy(mf.filter_bank(bank, [seg], 5.0, trig_cap=1 << 16)[0])
    bank.profile(True)
    got = mf.peaks_to_numpy(mf.filter_bank(bank, [seg], 5.0, trig_cap=1 << 16)[0])
    pr = bank.profile_read()
    bank.profile(False)
    assert bank.check() == 0
    assert np.array_equal(ref.view(np.uint8), got.view(np.uint8))
    N, n_t, n_b = spec.N, 64, 3
    assert pr["setup"][2] == 1 and pr["anchors"][2] == n_b and pr["pass1"][2] == n_b and pr["pass2"][2] == n_b
    assert all(pr[k][0] > 0 for k in ("setup", "anchors", "pass1", "pass2", "final"))
    assert pr["fused"][2] == 0
    assert pr["pass2"][1] == 8.0 * N * n_t
    band = sum(8.0 * (hi - lo) for lo, hi in (oracle.band(N, spec.fs, 40.0, min(oracle.f_isco(a, b), spec.fs / 2))
                                               for a, b in zip(wl.m1, wl.m2)))
    assert pr["pass1"][1] - pr["anchors"][1] == band + 8.0 * N * n_t
    assert pr["anchors"][1] > 0
    again = bank.profile_read()
    assert all(v == (0.0, 0.0, 0) for v in again.values())


def test_ragged_batches(mf, monkeypatch):
    """A bank size that is not a multiple of the templates in flight."""
    import torch
    wl = workloads.small(seed=4, N=1 << 13, fs=4096.0, n_templates=13)
    spec = wl.segments[0]
    s32, _ = oracle_segment(spec)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    bank = mf.Bank(wl.m1, wl.m2)
    ref = mf.peaks_to_numpy(mf.filter_bank(bank, [seg], 3.0, trig_cap=1 << 16)[0])
    monkeypatch.setenv("MFGB_BATCH", "5")
    got = mf.peaks_to_numpy(mf.filter_bank(bank, [seg], 3.0, trig_cap=1 << 16)[0])
    assert np.array_equal(ref.view(np.uint8), got.view(np.uint8))


def test_psd_table_and_scale(mf):
    """A caller PSD table: with the data fixed, S_n -> 3.7 S_n scales z by 1/3.7 and
    sigma by 1/sqrt(3.7), so rho -> rho/sqrt(3.7).  Data and PSD scaled together
    (physical units, S0 = 9e-46) leave rho unchanged."""
    import torch
    spec = workloads.small(seed=8, N=1 << 14).segments[0]
    s32, s64 = oracle_segment(spec)
    N, fs = spec.N, spec.fs
    bank = mf.Bank([1.5, 2.5], [1.4, 1.1])
    base = mf.peaks_to_numpy(mf.filter_bank(bank, [mf.Segment(torch.from_numpy(s32).cuda(), fs)], 100.0, 0)[0])
    S = oracle.psd_bins(N, fs) * 3.7
    S[0] = 1.0
    tab = mf.peaks_to_numpy(mf.filter_bank(bank, [mf.Segment(torch.from_numpy(s32).cuda(), fs, psd=S)], 100.0, 0)[0])
    assert np.max(np.abs(tab["rho"] * np.sqrt(3.7) - base["rho"]) / base["rho"]) < 1e-5
    assert np.array_equal(tab["j"], base["j"])
    phys = s32 * np.float32(3e-23)
    ph = mf.peaks_to_numpy(mf.filter_bank(bank, [mf.Segment(torch.from_numpy(phys).cuda(), fs, psd_S0=9e-46)],
                                          100.0, 0)[0])
    assert np.max(np.abs(ph["rho"] - base["rho"]) / base["rho"]) < 1e-4


@pytest.mark.parametrize("lg,fs,f_low", [(16, 4096.0, 40.0), (15, 2048.0, 30.0)])
def test_refine_matches_oracle(mf, lg, fs, f_low):
    """mf_refine_triggers: rho^2 and its gradient against the oracle's direct
    sum and analytic gradient (two sample rates and lower cut-offs)."""
    import torch
    N = 1 << lg
    spec = workloads.SegmentSpec(N, fs, 123)
    inj = np.zeros(1, dtype=oracle.INJ_DTYPE)
    inj[0] = (1.7, 1.3, 12.0, 5000, 0.4)
    spec.injections = inj
    s32, s64 = oracle_segment(spec, f_low)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), fs)
    t0 = ((N - 5000) % N) / fs
    theta = np.array([[1.7, 1.3, t0], [1.72, 1.31, t0 + 0.3 / fs], [1.65, 1.36, t0 - 1.7 / fs],
                      [2.5, 1.2, 1.0]])
    lo_hi = [oracle.band(N, fs, f_low, min(oracle.f_isco(a, b), fs / 2)) for a, b, _ in theta]
    ref_obj, ref_grad = oracle.refine(theta, s64, fs, f_low, bands=np.array(lo_hi))
    th = torch.tensor(theta, dtype=torch.float64, device="cuda")
    scale = np.abs(ref_grad).max(axis=0)
    for mode in (mf.MF_PHASE_FP64, mf.MF_PHASE_ANCHOR):     # per-bin FP64 phase, then the default anchors
        obj, grad = mf.refine(seg, th, f_low=f_low, phase_mode=mode)
        obj = obj.cpu().numpy()
        grad = grad.cpu().numpy()
        assert np.all(np.abs(obj - ref_obj) / np.maximum(ref_obj, 1.0) < REF_OBJ_TOL), (mode, obj, ref_obj)
        assert np.all(np.abs(grad - ref_grad) <= REF_GRAD_RTOL * np.abs(ref_grad) + REF_GRAD_ATOL * scale), (
            mode, grad, ref_grad)
    # explicit band gives the same as the default band at the same masses
    band = torch.tensor(np.array(lo_hi), dtype=torch.int64, device="cuda")
    obj2, grad2 = mf.refine(seg, th, band=band, f_low=f_low)
    assert np.array_equal(obj2.cpu().numpy(), obj)


def test_refine_autograd_function(mf):
    import torch
    N, fs = 1 << 14, 4096.0
    spec = workloads.SegmentSpec(N, fs, 7)
    inj = np.zeros(1, dtype=oracle.INJ_DTYPE)
    inj[0] = (1.5, 1.4, 15.0, 1000, 0.0)
    spec.injections = inj
    s32, _ = oracle_segment(spec)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), fs)
    theta = torch.tensor([[1.52, 1.39, ((N - 1000) % N) / fs + 0.2 / fs]], dtype=torch.float64,
                         device="cuda", requires_grad=True)
    J = mf.RefineFn.apply(theta, seg)
    (3.0 * J.sum()).backward()
    _, g = mf.refine(seg, theta.detach())
    assert torch.allclose(theta.grad, 3.0 * g)


def test_persistent_and_batch_schedulers_agree(mf, monkeypatch):
    """The persistent scheduler (one launch, ordered work queue) and the
    per-batch launches give bit-identical peaks and triggers."""
    import torch
    wl = workloads.small(seed=12, N=1 << 16, fs=4096.0, n_templates=21, m_lo=1.1, m_hi=9.0)
    spec = wl.segments[0]
    s32, _ = oracle_segment(spec)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    bank = mf.Bank(wl.m1, wl.m2)
    monkeypatch.setenv("MFGB_SCHED", "persistent")
    a = [x.cpu().numpy().copy() for x in mf.filter_bank(bank, [seg], 3.5, trig_cap=1 << 18)]
    monkeypatch.setenv("MFGB_SCHED", "batch")
    b = [x.cpu().numpy().copy() for x in mf.filter_bank(bank, [seg], 3.5, trig_cap=1 << 18)]
    assert int(a[2][0]) == int(b[2][0]) > 0
    n = int(a[2][0])
    assert np.array_equal(a[0].view(np.uint8), b[0].view(np.uint8))
    assert np.array_equal(a[1][:n].view(np.uint8), b[1][:n].view(np.uint8))


@pytest.mark.parametrize("lg,alt", [(19, 0), (20, 0), (21, 0), (22, 0), (20, 1), (22, 1)])
def test_pass2_rows_and_tiles_agree(mf, monkeypatch, lg, alt):
    """Pass 2 with whole rows per warp group (bulk-copy prefetch; rows of 1024
    points on one warp, 2048 on two, 4096 on four: the alternative splits of
    2^20 and 2^22) and the per-tile pass 2 give bit-identical peaks and
    triggers."""
    import torch
    wl = workloads.small(seed=40 + lg, N=1 << lg, fs=4096.0, n_templates=11, m_lo=1.1, m_hi=9.0)
    spec = wl.segments[0]
    s32, _ = oracle_segment(spec)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    bank = mf.Bank(wl.m1, wl.m2)
    monkeypatch.setenv("MFGB_SCHED", "batch")
    monkeypatch.setenv("MFGB_SPLIT_ALT", str(alt))
    monkeypatch.setenv("MFGB_BATCH", "4")          # ragged batches: 4 + 4 + 3
    a = [x.cpu().numpy().copy() for x in mf.filter_bank(bank, [seg], 3.5, trig_cap=1 << 20)]
    monkeypatch.setenv("MFGB_P2ROWS", "0")
    b = [x.cpu().numpy().copy() for x in mf.filter_bank(bank, [seg], 3.5, trig_cap=1 << 20)]
    assert bank.check() == 0
    n = int(a[2][0])
    assert int(b[2][0]) == n > 0
    assert np.array_equal(a[0].view(np.uint8), b[0].view(np.uint8))
    assert np.array_equal(a[1][:n].view(np.uint8), b[1][:n].view(np.uint8))


def test_bounded_wait_timeout_reports_and_recovers(mf, monkeypatch):
    """A wait of the persistent scheduler that can never be satisfied (test
    hook) runs out after its iteration limit: the call reports MF_ETIMEOUT,
    nothing faults, and the next call on the same bank is correct again."""
    import torch
    monkeypatch.setenv("MFGB_SCHED", "persistent")
    wl = workloads.small(seed=13, N=1 << 14, fs=4096.0, n_templates=6)
    spec = wl.segments[0]
    s32, _ = oracle_segment(spec)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    bank = mf.Bank(wl.m1, wl.m2)
    ref = mf.peaks_to_numpy(mf.filter_bank(bank, [seg], 4.0, trig_cap=1 << 16)[0])
    assert bank.check() == 0
    bank.debug_stall(3, spin_limit=2000)
    mf.filter_bank(bank, [seg], 4.0, trig_cap=1 << 16)
    assert bank.check(allow_timeout=True) == mf._native.MF_ETIMEOUT
    bank.debug_stall(-1)
    got = mf.peaks_to_numpy(mf.filter_bank(bank, [seg], 4.0, trig_cap=1 << 16)[0])
    assert bank.check() == 0
    assert np.array_equal(ref.view(np.uint8), got.view(np.uint8))


@pytest.mark.parametrize("lg", [19, 20])
def test_fused_scheduler_matches_batches_and_recovers(mf, monkeypatch, lg):
    """The fused scheduler (pass-1 CTAs and pass-2 warps in one launch, units
    streamed through a ring of exchange slots, here wrapped several times)
    gives peaks and triggers bit-identical to the per-batch launches; a
    dependency wait that can never be satisfied (test hook) runs out, the call
    reports MF_ETIMEOUT, nothing faults, and the next call is bit-identical."""
    import torch
    wl = workloads.small(seed=70 + lg, N=1 << lg, fs=4096.0, n_templates=37, m_lo=1.1, m_hi=6.0)
    spec = wl.segments[0]
    s32, _ = oracle_segment(spec)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    bank = mf.Bank(wl.m1, wl.m2)
    monkeypatch.setenv("MFGB_SCHED", "batch")
    a = [x.cpu().numpy().copy() for x in mf.filter_bank(bank, [seg], 5.0, trig_cap=1 << 18)]
    assert bank.check() == 0
    monkeypatch.setenv("MFGB_SCHED", "fused")
    for split in ("0.5", "0.7"):
        monkeypatch.setenv("MFGB_SPLIT", split)
        b = [x.cpu().numpy().copy() for x in mf.filter_bank(bank, [seg], 5.0, trig_cap=1 << 18)]
        assert bank.check() == 0
        n = int(a[2][0])
        assert int(b[2][0]) == n and n > 0
        assert np.array_equal(a[0].view(np.uint8), b[0].view(np.uint8))
        assert np.array_equal(a[1][:n].view(np.uint8), b[1][:n].view(np.uint8))
    monkeypatch.delenv("MFGB_SPLIT")
    bank.debug_stall(11, spin_limit=2000)
    mf.filter_bank(bank, [seg], 5.0, trig_cap=1 << 18)
    assert bank.check(allow_timeout=True) == mf._native.MF_ETIMEOUT
    bank.debug_stall(-1)
    c = [x.cpu().numpy().copy() for x in mf.filter_bank(bank, [seg], 5.0, trig_cap=1 << 18)]
    assert bank.check() == 0
    assert np.array_equal(a[0].view(np.uint8), c[0].view(np.uint8))
    assert np.array_equal(a[1][:int(a[2][0])].view(np.uint8), c[1][:int(a[2][0])].view(np.uint8))


@pytest.mark.parametrize("lg,fft,alt", [(20, "fp32", 0), (21, "fp32", 0), (22, "fp32", 1), (20, "tc_fp16", 0),
                                        (19, "tc_bf16", 0)])
def test_rows_kernel_timeout_reports_and_recovers(mf, monkeypatch, lg, fft, alt):
    """The per-batch rows kernels (1024-, 2048- and 4096-point rows, and the
    tensor-core form) with one template's row copies or MMA commits withheld
    (test hook): its waits run out, the call reports MF_ETIMEOUT, nothing
    faults, tensor memory is released, and the next call is bit-identical to
    one made before."""
    import torch
    monkeypatch.setenv("MFGB_SCHED", "batch")
    monkeypatch.setenv("MFGB_SPLIT_ALT", str(alt))
    fm = {"fp32": mf.MF_FFT_FP32, "tc_fp16": mf.MF_FFT_TC_FP16, "tc_bf16": mf.MF_FFT_TC_BF16}[fft]
    wl = workloads.small(seed=40 + lg, N=1 << lg, fs=4096.0, n_templates=5, m_lo=1.2, m_hi=6.0)
    spec = wl.segments[0]
    s32, _ = oracle_segment(spec)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    bank = mf.Bank(wl.m1, wl.m2, fft_mode=fm)
    a = [x.cpu().numpy().copy() for x in mf.filter_bank(bank, [seg], 5.0, trig_cap=1 << 18)]
    assert bank.check() == 0
    bank.debug_stall(2, spin_limit=2000)
    mf.filter_bank(bank, [seg], 5.0, trig_cap=1 << 18)
    assert bank.check(allow_timeout=True) == mf._native.MF_ETIMEOUT
    bank.debug_stall(-1)
    b = [x.cpu().numpy().copy() for x in mf.filter_bank(bank, [seg], 5.0, trig_cap=1 << 18)]
    assert bank.check() == 0
    n = int(a[2][0])
    assert int(b[2][0]) == n
    assert np.array_equal(a[0].view(np.uint8), b[0].view(np.uint8))
    assert np.array_equal(a[1][:n].view(np.uint8), b[1][:n].view(np.uint8))


def test_autotune_keeps_results(mf, tmp_path):
    """mf_autotune only changes the schedule: results stay bit-identical and
    the choice is written to the cache file."""
    import json
    import torch
    wl = workloads.small(seed=14, N=1 << 15, fs=4096.0, n_templates=9, m_lo=1.1, m_hi=6.0)
    spec = wl.segments[0]
    s32, _ = oracle_segment(spec)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    bank = mf.Bank(wl.m1, wl.m2)
    a = [x.cpu().numpy().copy() for x in mf.filter_bank(bank, [seg], 4.0, trig_cap=1 << 16)]
    cache = tmp_path / "tune.json"
    mf.autotune(bank, [seg], 4.0, repeats=1, cache_path=str(cache))
    rec = json.loads(cache.read_text())
    assert rec["scheduler"] in ("persistent", "batch") and rec["templates"] == 9
    assert rec["pass1"] in ("fused", "persistent-staged", "persistent-staged-half-tile", "per-tile")
    assert rec["pass2"] in ("fused", "rows", "per-tile")
    assert rec["n1_x_n2"]["32768"] in ("256 x 128", "128 x 256")   # no alternative split below 2^18
    assert rec["candidates"] >= 7
    b = [x.cpu().numpy().copy() for x in mf.filter_bank(bank, [seg], 4.0, trig_cap=1 << 16)]
    n = int(a[2][0])
    assert int(b[2][0]) == n
    assert np.array_equal(a[0].view(np.uint8), b[0].view(np.uint8))
    assert np.array_equal(a[1][:n].view(np.uint8), b[1][:n].view(np.uint8))
