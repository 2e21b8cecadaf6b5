"""Segment refresh and CUDA-graph capture of the bank filter (one graph launch
per step: conditioning of new samples, Eq. (1) weighting, and the filter of
Eqs. (1), (3), (4) over the bank).  Results of a replay must equal the eager
calls bit for bit: the graph only removes host launch work."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0906_4175_gb300 as m
    return m


def _two_segments(mf, N=1 << 16, fs=2048.0):
    import torch
    out = []
    for seed in (11, 12):
        inj = np.zeros(1, dtype=mf.INJ_DTYPE)
        inj[0] = (1.4, 1.4, 12.0, 3000 + 7 * seed, 0.3)
        spec = workloads.SegmentSpec(N=N, fs=fs, seed=seed, injections=inj)
        out.append(mf.synth_segment(spec.normals(), N, fs, 40.0, spec.injections))
    torch.cuda.synchronize()
    return out


def _filter(mf, bank, seg, thr, cap):
    p, t, n = mf.filter_bank(bank, [seg], thr, trig_cap=cap)
    return mf.peaks_to_numpy(p), mf.triggers_to_numpy(t, n), int(n.item())


def _same(a, b):
    assert a[2] == b[2]
    assert np.array_equal(a[0].view(np.uint8), b[0].view(np.uint8))
    assert np.array_equal(a[1].view(np.uint8), b[1].view(np.uint8))


def test_refresh_equals_upload(mf):
    s1, s2 = _two_segments(mf)
    rng = np.random.default_rng(3)
    m1 = rng.uniform(1.2, 1.6, 12)
    m2 = rng.uniform(1.2, 1.6, 12)
    bank = mf.Bank(m1, m2)
    ref2 = _filter(mf, bank, mf.Segment(s2, 2048.0), 5.0, 1 << 14)
    seg = mf.Segment(s1, 2048.0)
    seg.refresh(s2)                                  # device samples
    _same(_filter(mf, bank, seg, 5.0, 1 << 14), ref2)
    seg.refresh(s1.cpu().numpy())                    # host samples
    _same(_filter(mf, bank, seg, 5.0, 1 << 14), _filter(mf, bank, mf.Segment(s1, 2048.0), 5.0, 1 << 14))


def test_refresh_keeps_psd_table(mf):
    import torch
    s1, s2 = _two_segments(mf, N=1 << 14)
    f = np.arange((1 << 13) + 1) * (2048.0 / (1 << 14))
    x = np.maximum(f, 1.0) / 150.0
    psd = 2.5 * ((4.49 * x) ** -56 + 0.16 * x ** -4.52 + 0.52 + 0.32 * x * x)
    bank = mf.Bank([1.4, 1.3], [1.4, 1.5])
    ref = _filter(mf, bank, mf.Segment(s2, 2048.0, psd=psd), 4.0, 1 << 12)
    seg = mf.Segment(s1, 2048.0, psd=psd)
    seg.refresh(s2)
    torch.cuda.synchronize()
    _same(_filter(mf, bank, seg, 4.0, 1 << 12), ref)


@pytest.mark.parametrize("sched", ["persistent", "batch", "fused"])
def test_graph_replay_equals_eager(mf, monkeypatch, sched):
    import torch
    monkeypatch.setenv("MFGB_SCHED", sched)
    s1, s2 = _two_segments(mf)
    wl = workloads.tiny()
    bank = mf.Bank(wl.m1, wl.m2)
    cap = 1 << 14
    dev = torch.device("cuda", torch.cuda.current_device())
    s_buf = s1.clone()
    out = (torch.empty((bank.n, 4), dtype=torch.float32, device=dev),
           torch.empty((cap, 6), dtype=torch.float32, device=dev),
           torch.zeros(1, dtype=torch.int64, device=dev))
    seg = mf.Segment(s_buf, 2048.0)
    seg.refresh(s_buf)
    mf.filter_bank(bank, [seg], 5.0, trig_cap=cap, out=out)     # sizes the workspace
    torch.cuda.synchronize()
    l0 = mf.launch_count()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        seg.refresh(s_buf)
        mf.filter_bank(bank, [seg], 5.0, trig_cap=cap, out=out)
    per_replay = mf.launch_count() - l0
    assert per_replay >= 4
    for s in (s2, s1, s2):
        s_buf.copy_(s)
        g.replay()
        torch.cuda.synchronize()
        got = (mf.peaks_to_numpy(out[0]), mf.triggers_to_numpy(out[1], out[2]), int(out[2].item()))
        _same(got, _filter(mf, bank, mf.Segment(s, 2048.0), 5.0, cap))
    assert bank.check() == 0


def test_capture_refuses_workspace_growth(mf):
    import torch
    s1, _ = _two_segments(mf, N=1 << 14)
    bank = mf.Bank([1.4], [1.4])
    seg = mf.Segment(s1, 2048.0)
    mf.filter_bank(bank, [seg], 5.0, trig_cap=16)
    torch.cuda.synchronize()
    dev = torch.device("cuda", torch.cuda.current_device())
    out = (torch.empty((1, 4), dtype=torch.float32, device=dev),
           torch.empty((1 << 12, 6), dtype=torch.float32, device=dev),
           torch.zeros(1, dtype=torch.int64, device=dev))
    g = torch.cuda.CUDAGraph()
    err = None
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g.capture_begin()
        try:
            mf.filter_bank(bank, [seg], 5.0, trig_cap=1 << 12, out=out)   # larger trig_cap: must grow
        except mf.MFError as e:
            err = e
        finally:
            g.capture_end()
    assert err is not None and err.code == mf.MF_EINVAL
    # outside the capture the same call sizes the workspace and runs
    mf.filter_bank(bank, [seg], 5.0, trig_cap=1 << 12, out=out)
    torch.cuda.synchronize()
    assert bank.check() == 0
