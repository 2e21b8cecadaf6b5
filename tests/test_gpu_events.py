"""Events and per-event chi^2 through the C ABI against the oracle:
mf_cluster_triggers (two-stage single linkage; integer/index work, so
bit-exact on the same input records) and mf_chisq_points (Eq. 5 at single
samples by direct sums; the tolerance of test_gpu_chisq.py)."""
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


def _synthetic_triggers(seed, n_t, n_seg, N, per, rho_levels):
    """Seeded (tmpl, seg, j)-sorted trigger records with float32-exact values
    (rho from a few levels, so that ties occur)."""
    rng = np.random.default_rng(seed)
    rows = []
    for t in range(n_t):
        for s in range(n_seg):
            k = int(rng.integers(0, per))
            js = np.unique(rng.integers(0, N, k))
            for j in js:
                rows.append((t, s, int(j), float(rng.choice(rho_levels)), float(np.float32(rng.standard_normal())),
                             float(np.float32(rng.standard_normal()))))
    a = np.array(rows, dtype=[("tmpl", "i4"), ("seg", "i4"), ("j", "i4"), ("rho", "f4"), ("z_re", "f4"),
                              ("z_im", "f4")])
    return a[np.lexsort((a["j"], a["seg"], a["tmpl"]))]


def _to_oracle(a):
    o = np.zeros(a.size, dtype=oracle.TRIG_DTYPE)
    for f in ("tmpl", "seg", "j", "rho", "z_re", "z_im"):
        o[f] = a[f]
    return o


@pytest.mark.parametrize("seed,n_t,n_seg,N,per,W", [(1, 7, 3, 5000, 80, 0), (2, 7, 3, 5000, 80, 7),
                                                     (3, 40, 2, 1 << 16, 400, 64), (4, 300, 8, 1 << 20, 900, 4096),
                                                     (5, 3, 1, 1 << 12, 4000, 1)])
def test_cluster_matches_oracle_bit_exact(mf, seed, n_t, n_seg, N, per, W):
    import torch
    a = _synthetic_triggers(seed, n_t, n_seg, N, per, [6.0, 6.5, 7.25, 9.0, 12.5])
    cap = max(a.size, 1)
    t = torch.from_numpy(np.ascontiguousarray(a).view(np.float32).reshape(-1, 6).copy()).cuda()
    n = torch.tensor([a.size], dtype=torch.int64, device="cuda")
    ev, n_ev = mf.cluster_triggers(t, n, n_t, n_seg, N, W)
    got = mf.events_to_numpy(ev, n_ev)
    ref = oracle.cluster(_to_oracle(a), W)
    assert int(n_ev.item()) == ref.size
    for f in ("tmpl", "seg", "j", "n_trig", "n_tmpl"):
        assert np.array_equal(got[f], ref[f]), f
    assert np.array_equal(got["rho"], ref["rho"].astype(np.float32))
    assert np.array_equal(got["z_re"], ref["z_re"].astype(np.float32))
    assert int(got["n_trig"].sum()) == a.size


def test_cluster_truncates_and_empty(mf):
    import torch
    a = _synthetic_triggers(9, 5, 2, 4000, 60, [6.0, 7.0])
    t = torch.from_numpy(np.ascontiguousarray(a).view(np.float32).reshape(-1, 6).copy()).cuda()
    n = torch.tensor([a.size], dtype=torch.int64, device="cuda")
    ref = oracle.cluster(_to_oracle(a), 3)
    ev, n_ev = mf.cluster_triggers(t, n, 5, 2, 4000, 3, ev_cap=4)
    assert int(n_ev.item()) == ref.size > 4
    got = ev[:4].cpu().numpy().view(mf.EVENT_DTYPE).reshape(-1)
    assert np.array_equal(got["j"], ref["j"][:4])
    ev, n_ev = mf.cluster_triggers(t, torch.zeros(1, dtype=torch.int64, device="cuda"), 5, 2, 4000, 3)
    assert int(n_ev.item()) == 0


def test_events_of_tiny_workload(mf):
    """Filter -> cluster on the GPU against the oracle's filter -> cluster on the
    16-template, 2^16-sample case: the same events from the same triggers."""
    import torch
    wl = workloads.tiny(0)
    spec = wl.segments[0]
    s32, s64 = oracle_segment(spec)
    bank = mf.Bank(wl.m1, wl.m2)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    thr, W = 5.0, 2048
    p_, t_, n_ = mf.filter_bank(bank, [seg], thr, trig_cap=1 << 18)
    ev, n_ev = mf.cluster_triggers(t_, n_, bank.n, 1, spec.N, W)
    got = mf.events_to_numpy(ev, n_ev)
    _, otr, on, _ = oracle.filter_bank(wl.m1, wl.m2, s64, spec.fs, 40.0, thr)
    ref = oracle.cluster(otr, W)
    assert got.size == ref.size
    assert np.array_equal(got["j"], ref["j"]) and np.array_equal(got["tmpl"], ref["tmpl"])
    assert np.all(np.abs(got["rho"] - ref["rho"]) <= 1e-4 * ref["rho"])
    assert int(got["n_trig"].sum()) == int(n_.item()) == on


def test_chisq_points_match_oracle(mf):
    """Eq. (5) at chosen samples of two segments (2^14 and 2^15), rows in
    arbitrary order, including rows that name no template, segment or sample."""
    import torch
    rng = np.random.default_rng(21)
    m1, m2 = rng.uniform(1.2, 6.0, 6), rng.uniform(1.2, 6.0, 6)
    bank = mf.Bank(m1, m2)
    specs = [workloads.small(seed=70 + i, N=1 << lg, fs=4096.0, n_templates=1, m_lo=1.2, m_hi=6.0).segments[0]
             for i, lg in enumerate((14, 15))]
    data = [oracle_segment(sp) for sp in specs]
    segs = [mf.Segment(torch.from_numpy(d[0]).cuda(), sp.fs) for d, sp in zip(data, specs)]
    rows = []
    for _ in range(40):
        s = int(rng.integers(0, 2))
        rows.append((int(rng.integers(0, 6)), s, int(rng.integers(0, specs[s].N))))
    rows += [(6, 0, 5), (0, 2, 5), (0, 0, 1 << 20)]
    r = torch.tensor(np.array(rows, dtype=np.int32), device="cuda")
    got = mf.chisq_points(bank, segs, r, p=16).cpu().numpy().astype(np.float64)
    assert np.all(np.isnan(got[-3:]))
    cache = {}
    for i, (t, s, j) in enumerate(rows[:-3]):
        if (t, s) not in cache:
            chi, edges = mf.chisq_series(mf.Bank(m1[t:t + 1], m2[t:t + 1]), segs[s], [0], p=16)
            st, S = oracle.data_spectrum(data[s][1], specs[s].fs), oracle.psd_bins(specs[s].N, specs[s].fs)
            ref = oracle.chisq_series(float(m1[t]), float(m2[t]), st, S, specs[s].N, specs[s].fs, 40.0, 16)
            if not np.array_equal(ref["edges"], edges.cpu().numpy()[0]):
                assert np.max(np.abs(ref["edges"] - edges.cpu().numpy()[0])) <= 1
                ref = oracle.chisq_series(float(m1[t]), float(m2[t]), st, S, specs[s].N, specs[s].fs, 40.0, 16,
                                          edges=edges.cpu().numpy()[0])
            cache[(t, s)] = ref
        ref = cache[(t, s)]
        assert abs(got[i] - ref["chisq"][j]) <= chi2_tol(ref["chisq"][j], ref["rho"][j]), (i, t, s, j)
