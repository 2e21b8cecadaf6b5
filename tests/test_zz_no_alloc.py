"""mf_refine_triggers_static: the allocation-free variant of trigger refinement.

Callers that cannot allocate device memory while they refine (for example an
ascent loop running while another component owns the device allocator) use
this entry point; it keeps its partial sums in a fixed device array instead of
a stream allocation.  Its results must match mf_refine_triggers on the same
inputs, call after call, since the fixed array is reused and keeps the
previous call's contents.  Called through the C ABI directly.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from mfgb_testutil import oracle_segment

pytestmark = pytest.mark.gpu

OBJ_TOL = 2e-4   # relative, as in the refinement parity test


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


def _call(mf, fn, seg, theta, n):
    import torch
    obj = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    grad = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(seg.handle, None, ctypes.c_void_p(theta.data_ptr()), n, None, ctypes.c_void_p(obj.data_ptr()),
            ctypes.c_void_p(grad.data_ptr()), stream)
    assert rc == 0, mf._native.lib().mf_last_error()
    torch.cuda.synchronize()
    return obj.cpu().numpy(), grad.cpu().numpy()


def test_static_refine_matches_allocating_refine_twice(mf):
    import torch
    L = mf._native.lib()
    N, fs = 1 << 15, 4096.0
    spec = workloads.SegmentSpec(N, fs, 321)
    inj = np.zeros(1, dtype=oracle.INJ_DTYPE)
    inj[0] = (1.6, 1.3, 11.0, 7000, 0.2)
    spec.injections = inj
    s32, _ = oracle_segment(spec)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), fs)
    t0 = ((N - 7000) % N) / fs
    rng = np.random.default_rng(5)
    for call in range(2):
        n = 37 if call == 0 else 11          # second call: fewer rows, stale rows of call 1 remain in the array
        theta = np.column_stack([1.6 + rng.uniform(-0.05, 0.05, n), 1.3 + rng.uniform(-0.05, 0.05, n),
                                 t0 + rng.uniform(-3, 3, n) / fs])
        th = torch.tensor(theta, dtype=torch.float64, device="cuda")
        ref_obj, ref_grad = _call(mf, L.mf_refine_triggers, seg, th, n)
        got_obj, got_grad = _call(mf, L.mf_refine_triggers_static, seg, th, n)
        assert np.all(np.isfinite(got_obj)) and np.all(np.isfinite(got_grad))
        assert np.all(np.abs(got_obj - ref_obj) <= OBJ_TOL * np.maximum(np.abs(ref_obj), 1.0))
        scale = np.abs(ref_grad).max(axis=0)
        assert np.all(np.abs(got_grad - ref_grad) <= 2e-3 * np.abs(ref_grad) + 1e-4 * scale)


def test_static_refine_rejects_rows_beyond_its_scratch(mf):
    import torch
    L = mf._native.lib()
    N, fs = 1 << 12, 4096.0
    s32, _ = oracle_segment(workloads.SegmentSpec(N, fs, 5))
    seg = mf.Segment(torch.from_numpy(s32).cuda(), fs)
    n = 4097
    th = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    th[:, 0] = 1.4
    th[:, 1] = 1.4
    out = torch.zeros(n * 4, dtype=torch.float64, device="cuda")
    rc = L.mf_refine_triggers_static(seg.handle, None, ctypes.c_void_p(th.data_ptr()), n, None,
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(out.data_ptr() + 8 * n), None)
    assert rc == mf._native.MF_EINVAL
    assert b"4096" in L.mf_last_error()
