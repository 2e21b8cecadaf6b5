"""Parity of the CUDA path against the FP64 oracle on the three further
workloads of the method: an uneven bank over segments of several lengths in
one call (templates cut at their own ISCO frequency, Sec. 1.1), the precision
forms of the 2PN phase (Sec. 1.1 templates, Eq. 1 correlation), and gradient
refinement of coarse triggers (rho^2 of Eq. 3 at continuous t).

Tolerance: RHO_TOL = 1e-4 on err = |rho_gpu - rho_ref| / max(rho_ref, 1), as
in every parity test; indices exact unless the decision lies within RHO_TOL
of a tie or of the threshold."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import workloads
from mfgb_testutil import (REF_GRAD_ATOL, REF_GRAD_RTOL, REF_OBJ_TOL, RHO_TOL, oracle_segment, peak_index_agrees,
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


def _oracle_series(pairs, s64_by_seg, fs, f_low=40.0):
    """rho series of the oracle for (template index, m1, m2, segment) tuples,
    one ctypes call per thread (the oracle's C code runs without the GIL)."""
    cache = {}
    for si, s64 in s64_by_seg.items():
        N = s64.size
        cache[si] = (oracle.data_spectrum(s64, fs), oracle.psd_bins(N, fs), N)

    def one(p):
        t, a, b, si = p
        st, S, N = cache[si]
        return (t, si), oracle.filter_template(float(a), float(b), st, S, N, fs, f_low)["rho"]

    with ThreadPoolExecutor(max_workers=16) as ex:
        return dict(ex.map(one, pairs))


@pytest.fixture(scope="module")
def uneven_data(mf):
    import torch
    wl = workloads.uneven(0)
    s32, s64 = {}, {}
    for si, spec in enumerate(wl.segments):
        a, b = oracle_segment(spec)
        s32[si], s64[si] = a, b
    segs = [mf.Segment(torch.from_numpy(s32[si]).cuda(), spec.fs) for si, spec in enumerate(wl.segments)]
    return wl, s64, segs


def _uneven_call(mf, wl, segs, cap=1 << 22):
    bank = mf.Bank(wl.m1, wl.m2)
    p, t, n = mf.filter_bank(bank, segs, wl.threshold, trig_cap=cap)
    assert bank.check() == 0
    return bank, mf.peaks_to_numpy(p), mf.triggers_to_numpy(t, n), int(n.item())


def test_uneven_bank_against_oracle(mf, uneven_data):
    """4096 templates with M <= 35 (f_cut from 126 Hz to 2 kHz) over 8
    segments of 2^18..2^21 samples in ONE call; a sample of templates (the
    lightest, the heaviest, the loudest per segment, random ones) checked on
    every segment."""
    wl, s64, segs = uneven_data
    n_seg = len(segs)
    _, pk, tr, n = _uneven_call(mf, wl, segs)
    assert tr.size == n
    key = (tr["tmpl"].astype(np.int64) * n_seg + tr["seg"]) * (1 << 21) + tr["j"]
    assert np.all(np.diff(key) > 0)                       # sorted by (tmpl, seg, j)
    M = wl.m1 + wl.m2
    rho = pk["rho"].reshape(wl.n_templates, n_seg)
    loud = [int(np.argmax(rho[:, si])) for si in range(n_seg)]
    rng = np.random.default_rng(5)
    sample = sorted(set([int(np.argmin(M)), int(np.argmax(M))] + loud
                        + [int(x) for x in rng.choice(wl.n_templates, 6, replace=False)]))
    pairs = [(t, wl.m1[t], wl.m2[t], si) for t in sample for si in range(n_seg)]
    ref = _oracle_series(pairs, s64, wl.segments[0].fs)
    pk2 = pk.reshape(wl.n_templates, n_seg)
    for (t, si), r in ref.items():
        jr = int(np.argmax(r))
        assert peak_index_agrees(r, int(pk2[t, si]["j"]), jr), (t, si)
        assert abs(pk2[t, si]["rho"] - r[jr]) / max(1.0, r[jr]) <= RHO_TOL, (t, si)
    for si in range(n_seg):
        sel = tr[(tr["seg"] == si) & np.isin(tr["tmpl"], sample)]
        gk = {(int(a), int(b)) for a, b in zip(sel["tmpl"], sel["j"])}
        assert trigger_sets_agree(gk, {t: ref[(t, si)] for t in sample}, wl.threshold) == [], si
        for x in sel:
            r = ref[(int(x["tmpl"]), si)][x["j"]]
            assert abs(x["rho"] - r) / max(1.0, r) <= RHO_TOL
    # every injection is seen by some template of the bank in its segment
    assert all(rho[:, si].max() > wl.threshold for si in range(n_seg))


def test_uneven_bank_schedules_and_graph_agree(mf, uneven_data, monkeypatch):
    """The same uneven call under the persistent scheduler, the per-batch
    launches, per-template launches (first 256 templates) and one CUDA-graph
    replay gives bit-identical peaks and triggers."""
    import torch
    wl, _, segs = uneven_data
    monkeypatch.setenv("MFGB_SCHED", "persistent")
    monkeypatch.delenv("MFGB_BATCH", raising=False)
    _, pk_a, tr_a, n_a = _uneven_call(mf, wl, segs)
    monkeypatch.setenv("MFGB_SCHED", "batch")
    _, pk_b, tr_b, n_b = _uneven_call(mf, wl, segs)
    assert n_a == n_b
    assert np.array_equal(pk_a.view(np.uint8), pk_b.view(np.uint8))
    assert np.array_equal(tr_a.view(np.uint8), tr_b.view(np.uint8))
    # the fused scheduler (one launch per 2^19 / 2^20 segment, L2-resident exchange ring;
    # the other lengths fall back to per-batch launches)
    monkeypatch.setenv("MFGB_SCHED", "fused")
    _, pk_f, tr_f, n_f = _uneven_call(mf, wl, segs)
    assert n_f == n_a
    assert np.array_equal(pk_a.view(np.uint8), pk_f.view(np.uint8))
    assert np.array_equal(tr_a.view(np.uint8), tr_f.view(np.uint8))
    monkeypatch.setenv("MFGB_SCHED", "batch")
    # per-template launches on a prefix of the bank
    sub = workloads.Workload("prefix", wl.m1[:256], wl.m2[:256], wl.segments, threshold=wl.threshold)
    monkeypatch.setenv("MFGB_BATCH", "1")
    _, pk_c, tr_c, n_c = _uneven_call(mf, sub, segs)
    monkeypatch.delenv("MFGB_BATCH")
    monkeypatch.setenv("MFGB_SCHED", "persistent")
    _, pk_d, tr_d, n_d = _uneven_call(mf, sub, segs)
    assert n_c == n_d
    assert np.array_equal(pk_c.view(np.uint8), pk_d.view(np.uint8))
    assert np.array_equal(tr_c.view(np.uint8), tr_d.view(np.uint8))
    # one graph replay of the whole uneven call
    bank = mf.Bank(wl.m1, wl.m2)
    dev = torch.device("cuda", torch.cuda.current_device())
    cap = 1 << 22
    out = (torch.empty((bank.n * len(segs), 4), dtype=torch.float32, device=dev),
           torch.empty((cap, 6), dtype=torch.float32, device=dev),
           torch.zeros(1, dtype=torch.int64, device=dev))
    mf.filter_bank(bank, segs, wl.threshold, trig_cap=cap, out=out)
    torch.cuda.synchronize()
    out[0].zero_()
    out[2].zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        mf.filter_bank(bank, segs, wl.threshold, trig_cap=cap, out=out)
    g.replay()
    torch.cuda.synchronize()
    assert bank.check() == 0
    assert int(out[2].item()) == n_a
    assert np.array_equal(mf.peaks_to_numpy(out[0]).view(np.uint8), pk_a.view(np.uint8))
    assert np.array_equal(mf.triggers_to_numpy(out[1], out[2]).view(np.uint8), tr_a.view(np.uint8))


def test_uneven_bank_pass1_kernels_agree(mf, uneven_data, monkeypatch):
    """The persistent pass 1 (next tile staged by cp.async while the current
    one is transformed) and the per-tile pass 1 give bit-identical peaks and
    triggers on the uneven call (segments of 2^18 .. 2^21 samples)."""
    wl, _, segs = uneven_data
    monkeypatch.setenv("MFGB_SCHED", "batch")
    monkeypatch.setenv("MFGB_P1PF", "0")
    _, pk_a, tr_a, n_a = _uneven_call(mf, wl, segs)
    monkeypatch.setenv("MFGB_P1PF", "1")
    _, pk_b, tr_b, n_b = _uneven_call(mf, wl, segs)
    assert n_a == n_b
    assert np.array_equal(pk_a.view(np.uint8), pk_b.view(np.uint8))
    assert np.array_equal(tr_a.view(np.uint8), tr_b.view(np.uint8))
    # the persistent form with half-width column tiles (three CTAs per SM)
    monkeypatch.setenv("MFGB_P1TILE", "half")
    _, pk_c, tr_c, n_c = _uneven_call(mf, wl, segs)
    assert n_c == n_a
    assert np.array_equal(pk_a.view(np.uint8), pk_c.view(np.uint8))
    assert np.array_equal(tr_a.view(np.uint8), tr_c.view(np.uint8))
    # and staging W by per-thread cp.async instead of TMA (the form without a tensor map)
    monkeypatch.delenv("MFGB_P1TILE")
    monkeypatch.setenv("MFGB_P1TMA", "0")
    _, pk_d, tr_d, n_d = _uneven_call(mf, wl, segs)
    assert n_d == n_a
    assert np.array_equal(pk_a.view(np.uint8), pk_d.view(np.uint8))
    assert np.array_equal(tr_a.view(np.uint8), tr_d.view(np.uint8))


@pytest.mark.parametrize("sched", ["batch", "persistent", "fused"])
def test_uneven_bank_unit_order_agrees(mf, uneven_data, monkeypatch, sched):
    """Units run in descending band width (widest first); bank order gives
    bit-identical peaks and triggers under both schedulers, and the outputs
    stay in bank order (template t's peak in row t, whatever its position)."""
    wl, _, segs = uneven_data
    monkeypatch.setenv("MFGB_SCHED", sched)
    monkeypatch.setenv("MFGB_UNIT_ORDER", "bank")
    _, pk_a, tr_a, n_a = _uneven_call(mf, wl, segs)
    monkeypatch.delenv("MFGB_UNIT_ORDER")
    _, pk_b, tr_b, n_b = _uneven_call(mf, wl, segs)
    assert n_a == n_b
    assert np.array_equal(pk_a.view(np.uint8), pk_b.view(np.uint8))
    assert np.array_equal(tr_a.view(np.uint8), tr_b.view(np.uint8))


def _mode_errors(mf, wl, sample, s32, ref, phase_mode):
    """Full rho series of the sampled templates in one phase mode, compared
    with the oracle: (max err, median err, peak indices agree, trigger sets
    agree at the workload threshold)."""
    import torch
    spec = wl.segments[0]
    bank = mf.Bank(wl.m1[sample], wl.m2[sample], phase_mode=phase_mode)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    n_t = len(sample)
    p, t, n = mf.filter_bank(bank, [seg], 0.0, trig_cap=n_t * spec.N)
    assert bank.check() == 0
    tr = mf.triggers_to_numpy(t, n)
    rho = tr["rho"].reshape(n_t, spec.N).astype(np.float64)
    pk = mf.peaks_to_numpy(p)
    errs = np.concatenate([rho_err(rho[i], ref[i]) for i in range(n_t)])
    idx_ok = all(peak_index_agrees(ref[i], int(pk["j"][i]), int(np.argmax(ref[i]))) for i in range(n_t))
    gk = {(i, int(j)) for i in range(n_t) for j in np.nonzero(rho[i] > wl.threshold)[0]}
    trig_bad = trigger_sets_agree(gk, {i: ref[i] for i in range(n_t)}, wl.threshold)
    return float(errs.max()), float(np.median(errs)), idx_ok, trig_bad


def test_precision_forms_on_scale_bank(mf):
    """The 1024-template, N = 2^20 bank's data; 12 sampled templates (the two
    lightest, the two heaviest, the four loudest, random ones) in each phase
    form: FP64 anchors + FP32 Taylor (default) and FP64 per bin must meet
    RHO_TOL with exact indices; FP32-only phase is reported against them."""
    wl = workloads.scale(0)
    spec = wl.segments[0]
    s32, s64 = oracle_segment(spec)
    M = wl.m1 + wl.m2
    order = np.argsort(M)
    rng = np.random.default_rng(9)
    import torch
    bank = mf.Bank(wl.m1, wl.m2)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    pk = mf.peaks_to_numpy(mf.filter_bank(bank, [seg], wl.threshold, trig_cap=1 << 20)[0])
    loud = [int(x) for x in np.argsort(-pk["rho"])[:4]]
    sample = sorted(set([int(order[0]), int(order[1]), int(order[-1]), int(order[-2])] + loud
                        + [int(x) for x in rng.choice(wl.n_templates, 4, replace=False)]))
    pairs = [(i, wl.m1[t], wl.m2[t], 0) for i, t in enumerate(sample)]
    ref_d = _oracle_series(pairs, {0: s64}, spec.fs)
    ref = [ref_d[(i, 0)] for i in range(len(sample))]
    res = {}
    for name, mode in (("anchor", mf.MF_PHASE_ANCHOR), ("fp64", mf.MF_PHASE_FP64), ("fp32", mf.MF_PHASE_FP32)):
        res[name] = _mode_errors(mf, wl, sample, s32, ref, mode)
    for name in ("anchor", "fp64"):
        mx, med, idx_ok, bad = res[name]
        assert mx <= RHO_TOL, (name, mx)
        assert idx_ok, name
        assert bad == [], (name, bad[:5])
    # the FP32-only phase is the form the FP64 reduction exists to avoid
    assert res["fp32"][0] > res["anchor"][0], res
    print("precision forms (max, median rho err):",
          {k: (v[0], v[1], v[2], len(v[3])) for k, v in res.items()})


def coarse_triggers(tr, injections, N, fs, window_s=2.0):
    """Per injection, the loudest trigger within window_s of its coalescence
    sample (Eq. 1 read literally: a signal ending at j0 peaks at (N - j0) mod N)."""
    out = []
    for inj in injections:
        jc = (N - int(inj["j0"])) % N
        d = np.abs(((tr["j"].astype(np.int64) - jc + N // 2) % N) - N // 2)
        near = tr[d < int(window_s * fs)]
        if near.size:
            out.append((inj, near[np.argmax(near["rho"])]))
    return out


def ascend(mf, seg, theta0, steps=20, rel_m=5e-3, step_t=2e-4, row_seg=None):
    """Adam ascent of rho^2 on (m1, m2, t) through RefineFn.  The optimiser
    works on x = theta / scale (scale = rel_m * m for the masses, step_t for
    t), so one unit-rate Adam step moves each coordinate by about its scale.
    Returns the best point seen per row and its rho^2 (steps + 1 evaluations)."""
    import torch
    th0 = torch.as_tensor(theta0, dtype=torch.float64, device="cuda")
    sc = torch.stack([rel_m * th0[:, 0], rel_m * th0[:, 1], torch.full_like(th0[:, 2], step_t)], dim=1)
    x = (th0 / sc).clone().requires_grad_(True)
    opt = torch.optim.Adam([x], lr=1.0)
    best_th = th0.clone()
    best_J = torch.full((th0.shape[0],), -1.0, dtype=torch.float64, device="cuda")
    for k in range(steps + 1):
        th = x * sc
        J = mf.RefineFn.apply(th, seg, None, 40.0, row_seg)
        with torch.no_grad():
            better = J > best_J
            best_J = torch.where(better, J.detach(), best_J)
            best_th = torch.where(better[:, None], th.detach(), best_th)
        if k == steps:
            break
        opt.zero_grad()
        (-J.sum()).backward()
        opt.step()
    return best_th, best_J


def test_refinement_of_coarse_triggers(mf):
    """Coarse triggers of a 1-Msun bank (m in 1..20) on two N = 2^20 segments
    with 4 well separated injections each, refined by 20 Adam steps on
    (m1, m2, t) through RefineFn.  The refined rho^2 and its gradient at the
    end point equal the oracle's, and the refined rho^2 is never below the
    coarse trigger's."""
    import torch
    wl = workloads.refine_bank(0, n_segments=2, inj_per_segment=4)
    bank = mf.Bank(wl.m1, wl.m2)
    fs = wl.segments[0].fs
    for spec in wl.segments:
        s32, s64 = oracle_segment(spec)
        seg = mf.Segment(torch.from_numpy(s32).cuda(), fs)
        p, t, n = mf.filter_bank(bank, [seg], 4.0, trig_cap=1 << 22)
        assert bank.check() == 0
        tr = mf.triggers_to_numpy(t, n)
        N = spec.N
        found = coarse_triggers(tr, spec.injections, N, fs)
        assert len(found) >= 3
        theta0 = [[wl.m1[int(b["tmpl"])], wl.m2[int(b["tmpl"])], int(b["j"]) / fs] for _, b in found]
        rho0 = np.array([float(b["rho"]) for _, b in found])
        obj0, _ = mf.refine(seg, torch.tensor(theta0, dtype=torch.float64, device="cuda"))
        # the continuous-t objective at the coarse trigger is the filter's rho^2
        assert np.all(np.abs(np.sqrt(obj0.cpu().numpy()) - rho0) / rho0 < 2 * RHO_TOL)
        th, best = ascend(mf, seg, theta0)
        obj, grad = mf.refine(seg, th)
        assert np.array_equal(obj.cpu().numpy(), best.cpu().numpy())
        obj = obj.cpu().numpy()
        grad = grad.cpu().numpy()
        thn = th.cpu().numpy()
        lo_hi = [oracle.band(N, fs, 40.0, oracle.f_isco(a, b)) for a, b, _ in thn]
        ref_obj, ref_grad = oracle.refine(thn, s64, fs, 40.0, bands=np.array(lo_hi))
        assert np.all(np.abs(obj - ref_obj) / np.maximum(ref_obj, 1.0) < REF_OBJ_TOL), (obj, ref_obj)
        gs = np.abs(ref_grad).max(axis=0)
        assert np.all(np.abs(grad - ref_grad) <= REF_GRAD_RTOL * np.abs(ref_grad) + REF_GRAD_ATOL * gs)
        assert np.all(np.sqrt(obj) >= rho0 * (1 - 1e-4)), (np.sqrt(obj), rho0)


def test_refine_multi_segment_rows(mf):
    """mf_refine_triggers_multi: rows of three segments (two lengths) in one
    launch equal mf_refine_triggers on each row's own segment (to rounding of
    the grouped partial sums); a row naming no segment gets NaN."""
    import torch
    segs, thetas, rs = [], [], []
    for si, (lg, seed) in enumerate([(14, 1), (15, 2), (14, 3)]):
        N, fs = 1 << lg, 4096.0
        inj = np.zeros(1, dtype=oracle.INJ_DTYPE)
        inj[0] = (1.6 + 0.1 * si, 1.3, 14.0, 1000 + 77 * si, 0.2)
        spec = workloads.SegmentSpec(N, fs, 900 + seed, inj)
        s32, _ = oracle_segment(spec)
        segs.append(mf.Segment(torch.from_numpy(s32).cuda(), fs))
        t0 = ((N - int(inj[0]["j0"])) % N) / fs
        for d in (0.0, 0.4, -1.3):
            thetas.append([1.6 + 0.1 * si + 0.01 * d, 1.3, t0 + d / fs])
            rs.append(si)
    order = np.random.default_rng(4).permutation(len(rs))
    theta = torch.tensor(np.array(thetas)[order], dtype=torch.float64, device="cuda")
    row_seg = torch.tensor(np.array(rs, dtype=np.int32)[order], device="cuda")
    obj, grad = mf.refine(segs, theta, row_seg=row_seg)
    for si in range(3):
        sel = torch.nonzero(row_seg == si).flatten()
        o1, g1 = mf.refine(segs[si], theta[sel])
        # FP32 per-thread sums over differently grouped bins: agreement to FP32 rounding
        assert torch.allclose(obj[sel], o1, rtol=2e-5, atol=1e-6)
        assert torch.allclose(grad[sel], g1, rtol=1e-4, atol=1e-4 * float(g1.abs().max()))
    bad = row_seg.clone()
    bad[0] = 7
    ob, gb = mf.refine(segs, theta, row_seg=bad)
    assert torch.isnan(ob[0]) and torch.all(torch.isnan(gb[0]))
    assert torch.equal(ob[1:], obj[1:])


def test_refine_band_edges_outside_the_spectrum(mf):
    """A caller band whose edges lie beyond N/2 (or below 1) is clamped into
    [1, N/2] before the FP64 prefix P is read: a band starting beyond N/2 is
    empty (rho^2 = 0, zero gradient), one ending beyond N/2 equals the band
    ending at N/2, in every refinement entry point."""
    import ctypes
    import torch
    N, fs = 1 << 13, 4096.0
    s32, _ = oracle_segment(workloads.SegmentSpec(N, fs, 17))
    seg = mf.Segment(torch.from_numpy(s32).cuda(), fs)
    theta = torch.tensor([[1.5, 1.4, 0.3]] * 4, dtype=torch.float64, device="cuda")
    band = torch.tensor([[N // 2 + 5, N // 2 + 9], [N, 2 * N], [400, N // 2 + 100], [-50, 3000]],
                        dtype=torch.int64, device="cuda")
    clamped = torch.tensor([[N // 2, N // 2], [N // 2, N // 2], [400, N // 2], [1, 3000]],
                           dtype=torch.int64, device="cuda")
    obj, grad = mf.refine(seg, theta, band=band)
    ref, rgrad = mf.refine(seg, theta, band=clamped)
    assert torch.equal(obj, ref) and torch.equal(grad, rgrad)
    assert float(obj[0]) == 0.0 and float(obj[1]) == 0.0 and torch.all(grad[:2] == 0)
    assert float(obj[2]) > 0.0 and float(obj[3]) > 0.0
    row_seg = torch.zeros(4, dtype=torch.int32, device="cuda")
    om, gm = mf.refine([seg], theta, band=band, row_seg=row_seg)
    assert torch.equal(om[:2], obj[:2]) and torch.allclose(om, obj, rtol=2e-5, atol=1e-6)
    L = mf._native.lib()
    os_ = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    gs = torch.full((4, 3), float("nan"), dtype=torch.float64, device="cuda")
    rc = L.mf_refine_triggers_static(seg.handle, None, ctypes.c_void_p(theta.data_ptr()), 4,
                                     ctypes.c_void_p(band.data_ptr()), ctypes.c_void_p(os_.data_ptr()),
                                     ctypes.c_void_p(gs.data_ptr()), None)
    assert rc == 0, L.mf_last_error()
    torch.cuda.synchronize()
    assert torch.equal(os_[:2], obj[:2]) and torch.allclose(os_, obj, rtol=2e-5, atol=1e-6)
