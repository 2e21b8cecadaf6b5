"""The debug build's index checks (mf_debug_status): the library compiled with
MFGB_DEBUG range-checks the computed indices of the exchange stores and
loads, the anchor records, the TMA and bulk copies, the row kernels, the
persistent scheduler's queue items and the trigger sort's scatter, skipping an
access that fails and setting a status bit.  Every form of the filter runs
under it with the status word zero and outputs equal to the release build's.
No case is made to go out of range on purpose."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, N, fs, n_templates, environment of the call)
CASES = [
    ("n12", 1 << 12, 4096.0, 5, {}),
    ("n16_batch", 1 << 16, 4096.0, 9, {"MFGB_SCHED": "batch"}),
    ("n16_persistent", 1 << 16, 4096.0, 9, {"MFGB_SCHED": "persistent"}),
    ("n18_alt_split", 1 << 18, 4096.0, 5, {"MFGB_SCHED": "batch", "MFGB_SPLIT_ALT": "1"}),
    ("n20_staged", 1 << 20, 4096.0, 6, {"MFGB_SCHED": "batch", "MFGB_BATCH": "4"}),
    ("n20_half_tile", 1 << 20, 4096.0, 6, {"MFGB_SCHED": "batch", "MFGB_P1TILE": "half"}),
    ("n20_cpasync_pertile_p2", 1 << 20, 4096.0, 6, {"MFGB_SCHED": "batch", "MFGB_P1TMA": "0", "MFGB_P2ROWS": "0"}),
    ("n20_persistent", 1 << 20, 4096.0, 6, {"MFGB_SCHED": "persistent"}),
    ("n19_fused", 1 << 19, 4096.0, 7, {"MFGB_SCHED": "fused"}),
    ("n20_fused", 1 << 20, 4096.0, 6, {"MFGB_SCHED": "fused"}),
    ("n21", 1 << 21, 4096.0, 3, {"MFGB_SCHED": "batch"}),
    ("n22", 1 << 22, 4096.0, 2, {"MFGB_SCHED": "batch"}),
    ("n22_alt_split", 1 << 22, 4096.0, 2, {"MFGB_SCHED": "batch", "MFGB_SPLIT_ALT": "1"}),
]

CHILD = r'''
import ctypes, os, sys
import numpy as np, torch
sys.path.insert(0, ROOT); sys.path.insert(0, os.path.join(ROOT, "tests"))
import paper_0906_4175_gb300 as mf, workloads
out = {}
L = mf._native.lib()
for name, N, fs, nt, env in CASES:
    for k in ("MFGB_SCHED", "MFGB_SPLIT_ALT", "MFGB_BATCH", "MFGB_P1TILE", "MFGB_P1TMA", "MFGB_P2ROWS"):
        os.environ.pop(k, None)
    os.environ.update(env)
    wl = workloads.small(seed=N % 997 + nt, N=N, fs=fs, n_templates=nt, m_lo=1.1, m_hi=7.0, snr=20.0)
    sp = wl.segments[0]
    s = mf.synth_segment(sp.normals(), sp.N, sp.fs, wl.f_low, sp.injections)
    bank = mf.Bank(wl.m1, wl.m2)
    seg = mf.Segment(s, sp.fs)
    p, t, n = mf.filter_bank(bank, [seg], 5.0, trig_cap=1 << 16)
    bank.check()
    out[name + "_peaks"] = mf.peaks_to_numpy(p)
    out[name + "_trig"] = mf.triggers_to_numpy(t, n)
    if name == "n20_staged":   # chi^2 rows kernel (bulk-copied sub-band rows) on the same bank
        chi, edges = mf.chisq_series(bank, seg, torch.arange(2, dtype=torch.int32, device="cuda"), p=4)
        out["chisq"] = chi.cpu().numpy()
        out["edges"] = edges.cpu().numpy()
    if name in ("n20_staged", "n19_fused"):   # p = 16: sub-bands narrow enough for the single-row first stage
        chi, edges = mf.chisq_series(bank, seg, torch.arange(2, dtype=torch.int32, device="cuda"), p=16)
        out[name + "_chisq16"] = chi.cpu().numpy()
        out[name + "_edges16"] = edges.cpu().numpy()
w = ctypes.c_uint32(); en = ctypes.c_int()
assert L.mf_debug_status(ctypes.byref(w), ctypes.byref(en)) == 0
out["status"] = np.array([w.value, en.value])
np.savez(OUT, **out)
'''


def _run(tmp_path, debug):
    out = tmp_path / ("debug.npz" if debug else "release.npz")
    env = dict(os.environ)
    env["MFGB_DEBUG_LIB"] = "1" if debug else "0"
    code = "ROOT = %r\nOUT = %r\nCASES = %r\n" % (ROOT, str(out), CASES) + CHILD
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(out)


def test_debug_build_index_checks_stay_clear(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_4175_gb300 import build
    build.build()
    build.build(debug=True)
    dbg = _run(tmp_path, True)
    rel = _run(tmp_path, False)
    assert int(dbg["status"][1]) == 1 and int(rel["status"][1]) == 0   # the debug library was the one loaded
    assert int(dbg["status"][0]) == 0, "debug index checks failed: bits 0x%x" % int(dbg["status"][0])
    for k in rel.files:
        if k != "status":
            assert np.array_equal(dbg[k].view(np.uint8), rel[k].view(np.uint8)), k
