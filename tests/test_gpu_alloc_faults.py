"""Host-side fault injection for device allocations (mf_debug_fail_alloc).

For each entry point that allocates device memory, every one of its
allocations is made to fail in turn (countdown 0, 1, 2, ... until the call
goes through): each failing call must return MF_ENOMEM without faulting,
and the handles it was given must stay usable, so that the call that finally
succeeds -- and later calls -- give results bit-identical to a run without
injected faults.  The fault is made on the host (the allocation is never
attempted); no GPU fault or hang is involved.
"""
import numpy as np
import pytest

import oracle
import workloads
from mfgb_testutil import oracle_segment

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


def _sweep(mf, fn, max_allocs=64):
    """Run fn() with the k-th device allocation failing, k = 0, 1, ...; every
    failing run must raise MF_ENOMEM.  Returns (allocations fn makes, the
    result of the run that went through)."""
    L = mf._native.lib()
    for k in range(max_allocs):
        L.mf_debug_fail_alloc(k)
        try:
            out = fn()
        except mf._native.MFError as e:
            assert e.code == mf._native.MF_ENOMEM, (k, str(e))
            assert "memory" in str(e), str(e)
            continue
        finally:
            L.mf_debug_fail_alloc(-1)
        return k, out
    raise AssertionError("the call never went through")


def _np(xs):
    return [x.cpu().numpy().copy() for x in xs]


def _same(a, b):
    n = int(a[2][0])
    assert int(b[2][0]) == n
    assert np.array_equal(a[0].view(np.uint8), b[0].view(np.uint8))
    assert np.array_equal(a[1][:n].view(np.uint8), b[1][:n].view(np.uint8))


def test_filter_path_allocation_failures(mf):
    """Bank and segment creation, the first filter call of a bank (workspace
    growth), a regrowth for a longer segment, the first refresh of a segment
    from host samples."""
    import torch
    wl = workloads.small(seed=5, N=1 << 16, fs=4096.0, n_templates=6, m_lo=1.2, m_hi=5.0)
    wl2 = workloads.small(seed=6, N=1 << 18, fs=4096.0, n_templates=6, m_lo=1.2, m_hi=5.0)
    s1, _ = oracle_segment(wl.segments[0])
    s2, _ = oracle_segment(wl2.segments[0])
    fs = wl.segments[0].fs
    ref_bank = mf.Bank(wl.m1, wl.m2)
    ref_seg1 = mf.Segment(torch.from_numpy(s1).cuda(), fs)
    ref_seg2 = mf.Segment(torch.from_numpy(s2).cuda(), fs)
    ref1 = _np(mf.filter_bank(ref_bank, [ref_seg1], 4.0, trig_cap=1 << 16))
    ref2 = _np(mf.filter_bank(ref_bank, [ref_seg2], 4.0, trig_cap=1 << 16))

    n, bank = _sweep(mf, lambda: mf.Bank(wl.m1, wl.m2))
    assert n >= 2
    n, seg1 = _sweep(mf, lambda: mf.Segment(s1, fs))            # host samples: upload copies them
    assert n >= 5
    seg2 = mf.Segment(torch.from_numpy(s2).cuda(), fs)
    n, out = _sweep(mf, lambda: _np(mf.filter_bank(bank, [seg1], 4.0, trig_cap=1 << 16)))
    assert n >= 10                                                 # the bank's workspace
    _same(ref1, out)
    n, out = _sweep(mf, lambda: _np(mf.filter_bank(bank, [seg2], 4.0, trig_cap=1 << 16)))
    assert n >= 10                                                 # regrown for 2^18
    _same(ref2, out)
    _same(ref1, _np(mf.filter_bank(bank, [seg1], 4.0, trig_cap=1 << 16)))
    assert bank.check() == 0
    # first refresh from host samples: its conditioning buffers
    seg3 = mf.Segment(torch.from_numpy(s1).cuda(), fs)
    n, _ = _sweep(mf, lambda: seg3.refresh(s1))
    assert n >= 2
    _same(ref1, _np(mf.filter_bank(bank, [seg3], 4.0, trig_cap=1 << 16)))


def test_search_tail_allocation_failures(mf):
    """chi^2 series, trigger clustering, refinement (single and multi-segment),
    segment synthesis and the batched FFT."""
    import torch
    wl = workloads.small(seed=8, N=1 << 16, fs=4096.0, n_templates=5, m_lo=1.2, m_hi=4.0, snr=20.0)
    spec = wl.segments[0]
    s32, _ = oracle_segment(spec)
    bank = mf.Bank(wl.m1, wl.m2)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    peaks, trig, n_trig = mf.filter_bank(bank, [seg], 5.0, trig_cap=1 << 16)
    tmpl = torch.arange(3, dtype=torch.int32, device="cuda")

    ref = mf.chisq_series(bank, seg, tmpl, p=4)
    n, got = _sweep(mf, lambda: mf.chisq_series(bank, seg, tmpl, p=4))
    assert n >= 3
    for a, b in zip(ref, got):
        assert torch.equal(a, b)

    ref = mf.cluster_triggers(trig, n_trig, bank.n, 1, spec.N, 4096)
    n, got = _sweep(mf, lambda: mf.cluster_triggers(trig, n_trig, bank.n, 1, spec.N, 4096))
    assert n >= 5
    ne = int(ref[1].item())
    assert int(got[1].item()) == ne
    assert torch.equal(ref[0][:ne], got[0][:ne])

    pk = mf.peaks_to_numpy(peaks)
    theta = torch.tensor(np.column_stack([wl.m1, wl.m2, ((spec.N - pk["j"]) % spec.N) / spec.fs]),
                         dtype=torch.float64, device="cuda")
    ref = mf.refine(seg, theta)
    n, got = _sweep(mf, lambda: mf.refine(seg, theta))
    assert n >= 1
    assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1])
    rows = torch.zeros(theta.shape[0], dtype=torch.int32, device="cuda")
    ref = mf.refine([seg], theta, row_seg=rows)
    n, got = _sweep(mf, lambda: mf.refine([seg], theta, row_seg=rows))
    assert n >= 1
    assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1])

    g = spec.normals()
    ref = mf.synth_segment(g, spec.N, spec.fs, 40.0, spec.injections)
    n, got = _sweep(mf, lambda: mf.synth_segment(g, spec.N, spec.fs, 40.0, spec.injections))
    assert n >= 3
    assert torch.equal(ref, got)

    x = torch.randn(4, 1 << 14, dtype=torch.complex64, device="cuda")
    ref = mf.fft(x)
    n, got = _sweep(mf, lambda: mf.fft(x))
    assert torch.equal(ref, got)
