"""Tensor-core DFT stage (fft_mode MF_FFT_TC_FP16 / MF_FFT_TC_BF16): the first
radix-32 stage of the 1024-point rows of pass 2 as hi + lo split products on
the tensor cores (tcgen05.mma, FP32 accumulate), everything else FP32.

Both forms are held to the FP32 path's bound, RHO_TOL = 1e-4 on
err_j = |rho_gpu - rho_ref| / max(rho_ref, 1) against the FP64 oracle, with
peak and trigger indices exact wherever the decision is not within RHO_TOL of
a tie or of the threshold.  (The split products of one DFT-32 stage are good
to about 3e-6 (BF16) and 1e-6 (FP16) of the stage's largest output; the bench's
precision workload reports the resulting rho errors.)"""
import numpy as np
import pytest

import oracle
import workloads
from mfgb_testutil import (RHO_TOL, gpu_rho_series, oracle_rho_series, oracle_segment, peak_index_agrees,
                           rho_err, trigger_sets_agree)

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


@pytest.mark.parametrize("mode", ["fp16", "bf16"])
@pytest.mark.parametrize("lg", [19, 20])
def test_tc_forms_full_series(mf, lg, mode):
    """Every rho_j and z_j of four templates (M from 2.4 to 24 Msun: bands cut
    far below Nyquist) at N = 2^19 and 2^20 against the oracle."""
    import torch
    fm = mf.MF_FFT_TC_FP16 if mode == "fp16" else mf.MF_FFT_TC_BF16
    wl = workloads.small(seed=300 + lg, N=1 << lg, fs=4096.0, n_templates=4, m_lo=1.2, m_hi=12.0)
    spec = wl.segments[0]
    s32, s64 = oracle_segment(spec)
    bank = mf.Bank(wl.m1, wl.m2, fft_mode=fm)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    rho_g, z_g, peaks = gpu_rho_series(mf, bank, seg, len(wl.m1), spec.N)
    ref = oracle_rho_series(wl.m1, wl.m2, s64, spec.fs)
    for t, r in enumerate(ref):
        e = rho_err(rho_g[t], r["rho"])
        assert e.max() <= RHO_TOL, (t, float(e.max()))
        jr = int(np.argmax(r["rho"]))
        assert peak_index_agrees(r["rho"], int(peaks["j"][t]), jr), (t, peaks["j"][t], jr)
        ez = np.abs(z_g[t] - r["z"]) / r["sigma"]
        assert ez.max() <= RHO_TOL, (t, float(ez.max()))


@pytest.mark.parametrize("mode", ["fp16", "bf16"])
def test_tc_forms_on_bench_bank(mf, mode):
    """64 templates of the 1024-template bench bank on its 2^20-sample segment
    with 8 injections: peaks and triggers of the tensor-core form against the
    FP32 form, and the four loudest templates against the oracle."""
    import torch
    fm = mf.MF_FFT_TC_FP16 if mode == "fp16" else mf.MF_FFT_TC_BF16
    wl = workloads.scale(0)
    spec = wl.segments[0]
    s32, s64 = oracle_segment(spec)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    sel = np.arange(0, 1024, 16)
    out = {}
    for name, f in (("fp32", mf.MF_FFT_FP32), ("tc", fm)):
        bank = mf.Bank(wl.m1[sel], wl.m2[sel], fft_mode=f)
        peaks, trig, n = mf.filter_bank(bank, [seg], wl.threshold, trig_cap=1 << 20)
        assert bank.check() == 0
        out[name] = (mf.peaks_to_numpy(peaks), mf.triggers_to_numpy(trig, n))
    pa, ta = out["fp32"]
    pb, tb = out["tc"]
    assert np.all(np.abs(pa["rho"] - pb["rho"]) / np.maximum(pa["rho"], 1.0) <= RHO_TOL)
    loud = [int(x) for x in np.argsort(-pa["rho"])[:4]]
    ref = oracle_rho_series(wl.m1[sel][loud], wl.m2[sel][loud], s64, spec.fs)
    for i, t in enumerate(loud):
        r = ref[i]["rho"]
        jr = int(np.argmax(r))
        assert peak_index_agrees(r, int(pb["j"][t]), jr), (t, pb["j"][t], jr)
        assert abs(pb["rho"][t] - r[jr]) / max(r[jr], 1.0) <= RHO_TOL
        gk = {(t, int(j)) for j in tb["j"][tb["tmpl"] == t]}
        assert trigger_sets_agree(gk, {t: r}, wl.threshold) == [], t
    # the two forms' trigger sets differ only within RHO_TOL of the threshold
    ka = {(int(a), int(b)): float(c) for a, b, c in zip(ta["tmpl"], ta["j"], ta["rho"])}
    kb = {(int(a), int(b)): float(c) for a, b, c in zip(tb["tmpl"], tb["j"], tb["rho"])}
    for k in set(ka) ^ set(kb):
        r = ka.get(k, kb.get(k))
        assert abs(r - wl.threshold) / wl.threshold <= RHO_TOL, (k, r)


def test_tc_forms_reject_other_lengths(mf):
    """The tensor-core stage exists for 1024-point rows only: N = 2^18 and
    2^21 return MF_ENOTSUP; an unknown fft_mode is refused at bank creation."""
    import torch
    for lg in (18, 21):
        bank = mf.Bank([1.4], [1.4], fft_mode=mf.MF_FFT_TC_BF16)
        seg = mf.Segment(torch.zeros(1 << lg, device="cuda"), 4096.0)
        with pytest.raises(mf.MFError) as ei:
            mf.filter_bank(bank, [seg], 6.0)
        assert "MF_ENOTSUP" in str(ei.value)
    with pytest.raises(mf.MFError) as ei:
        mf.Bank([1.4], [1.4], fft_mode=3)
    assert "MF_ENOTSUP" in str(ei.value)
