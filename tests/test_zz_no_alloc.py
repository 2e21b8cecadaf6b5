"""mf_refine_triggers_static: the allocation-free variant of trigger refinement.

Callers that cannot allocate device memory while they refine (for example an
ascent loop running while another component owns the device allocator) use
this entry point; it keeps its partial sums in a fixed device array instead of
a stream allocation.  Its results must match mf_refine_triggers on the same
inputs, call after call, since the fixed array is reused and keeps the
previous call's contents; they must match the FP64 oracle as the allocating
path does; and a call must not draw on the device's stream-ordered memory
pool at all.  Called through the C ABI directly.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from mfgb_testutil import REF_GRAD_ATOL, REF_GRAD_RTOL, REF_OBJ_TOL, oracle_segment

pytestmark = pytest.mark.gpu

MAX_ROWS = 4096  # the entry point's fixed scratch holds this many rows

CU_MEMPOOL_ATTR_USED_MEM_CURRENT = 7
CU_MEMPOOL_ATTR_USED_MEM_HIGH = 8


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


class PoolWatch:
    """Used-memory figures of the current device's stream-ordered memory pool
    (the pool cudaMallocAsync draws from), read through the driver API."""

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetMemPool(ctypes.byref(self.pool), dev) == 0

    def _get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)   # resets the high-water mark to the current use
        assert self.cu.cuMemPoolSetAttribute(self.pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH, ctypes.byref(zero)) == 0

    def current(self):
        return self._get(CU_MEMPOOL_ATTR_USED_MEM_CURRENT)

    def high(self):
        return self._get(CU_MEMPOOL_ATTR_USED_MEM_HIGH)


def _outputs(n):
    import torch
    obj = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    grad = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    return obj, grad


def _launch(mf, fn, seg, theta, n, obj, grad):
    import torch
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(seg.handle, None, ctypes.c_void_p(theta.data_ptr()), n, None, ctypes.c_void_p(obj.data_ptr()),
            ctypes.c_void_p(grad.data_ptr()), stream)
    assert rc == 0, mf._native.lib().mf_last_error()


def _call(mf, fn, seg, theta, n):
    import torch
    obj, grad = _outputs(n)
    _launch(mf, fn, seg, theta, n, obj, grad)
    torch.cuda.synchronize()
    return obj.cpu().numpy(), grad.cpu().numpy()


def _segment(mf, N, fs, seed, j0):
    import torch
    spec = workloads.SegmentSpec(N, fs, seed)
    inj = np.zeros(1, dtype=oracle.INJ_DTYPE)
    inj[0] = (1.6, 1.3, 11.0, j0, 0.2)
    spec.injections = inj
    s32, s64 = oracle_segment(spec)
    return mf.Segment(torch.from_numpy(s32).cuda(), fs), s64


def _theta(rng, n, t0, fs):
    return np.column_stack([1.6 + rng.uniform(-0.05, 0.05, n), 1.3 + rng.uniform(-0.05, 0.05, n),
                            t0 + rng.uniform(-3, 3, n) / fs])


def _assert_close(got_obj, got_grad, ref_obj, ref_grad):
    assert np.all(np.isfinite(got_obj)) and np.all(np.isfinite(got_grad))
    assert np.all(np.abs(got_obj - ref_obj) <= REF_OBJ_TOL * np.maximum(np.abs(ref_obj), 1.0))
    scale = np.abs(ref_grad).max(axis=0)
    assert np.all(np.abs(got_grad - ref_grad) <= REF_GRAD_RTOL * np.abs(ref_grad) + REF_GRAD_ATOL * scale)


def test_static_refine_matches_allocating_refine_and_oracle_twice(mf):
    import torch
    L = mf._native.lib()
    N, fs = 1 << 15, 4096.0
    seg, s64 = _segment(mf, N, fs, 321, 7000)
    t0 = ((N - 7000) % N) / fs
    rng = np.random.default_rng(5)
    for call in range(2):
        n = 37 if call == 0 else 11          # second call: fewer rows, stale rows of call 1 remain in the array
        theta = _theta(rng, n, t0, fs)
        th = torch.tensor(theta, dtype=torch.float64, device="cuda")
        ref_obj, ref_grad = _call(mf, L.mf_refine_triggers, seg, th, n)
        got_obj, got_grad = _call(mf, L.mf_refine_triggers_static, seg, th, n)
        _assert_close(got_obj, got_grad, ref_obj, ref_grad)
        bands = np.array([oracle.band(N, fs, 40.0, oracle.f_isco(a, b)) for a, b, _ in theta])
        or_obj, or_grad = oracle.refine(theta, s64, fs, 40.0, bands=bands)
        _assert_close(got_obj, got_grad, or_obj, or_grad)


def test_static_refine_full_scratch(mf):
    """n = 4096, the largest call: the row records then end exactly at the end
    of the fixed array.  Every row equals the allocating path's, and a seeded
    sample of rows equals the oracle's."""
    import torch
    L = mf._native.lib()
    N, fs = 1 << 14, 4096.0
    seg, s64 = _segment(mf, N, fs, 77, 3000)
    t0 = ((N - 3000) % N) / fs
    rng = np.random.default_rng(11)
    theta = _theta(rng, MAX_ROWS, t0, fs)
    th = torch.tensor(theta, dtype=torch.float64, device="cuda")
    got_obj, got_grad = _call(mf, L.mf_refine_triggers_static, seg, th, MAX_ROWS)
    ref_obj, ref_grad = _call(mf, L.mf_refine_triggers, seg, th, MAX_ROWS)
    _assert_close(got_obj, got_grad, ref_obj, ref_grad)
    pick = np.sort(rng.choice(MAX_ROWS, 64, replace=False))
    bands = np.array([oracle.band(N, fs, 40.0, oracle.f_isco(a, b)) for a, b, _ in theta[pick]])
    or_obj, or_grad = oracle.refine(theta[pick], s64, fs, 40.0, bands=bands)
    _assert_close(got_obj[pick], got_grad[pick], or_obj, or_grad)


def test_static_refine_draws_nothing_from_the_memory_pool(mf):
    """Across a call (after the first on this device) the stream-ordered pool's
    used memory and its high-water mark stay where they were, while the
    allocating entry point on the same rows raises the high-water mark: the
    watch sees a stream allocation when there is one."""
    import torch
    L = mf._native.lib()
    N, fs = 1 << 13, 4096.0
    seg, _ = _segment(mf, N, fs, 9, 1000)
    t0 = ((N - 1000) % N) / fs
    n = 256
    th = torch.tensor(_theta(np.random.default_rng(2), n, t0, fs), dtype=torch.float64, device="cuda")
    obj, grad = _outputs(n)
    _launch(mf, L.mf_refine_triggers_static, seg, th, n, obj, grad)   # first call: symbol look-up
    torch.cuda.synchronize()
    watch = PoolWatch()
    watch.reset_high()
    before = watch.current()
    assert watch.high() == before
    for _ in range(3):
        _launch(mf, L.mf_refine_triggers_static, seg, th, n, obj, grad)
    torch.cuda.synchronize()
    assert watch.current() == before and watch.high() == before
    _launch(mf, L.mf_refine_triggers, seg, th, n, obj, grad)
    torch.cuda.synchronize()
    assert watch.high() > before
    assert watch.current() == before


def test_static_refine_rejects_rows_beyond_its_scratch(mf):
    import torch
    L = mf._native.lib()
    N, fs = 1 << 12, 4096.0
    s32, _ = oracle_segment(workloads.SegmentSpec(N, fs, 5))
    seg = mf.Segment(torch.from_numpy(s32).cuda(), fs)
    n = MAX_ROWS + 1
    th = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    th[:, 0] = 1.4
    th[:, 1] = 1.4
    out = torch.zeros(n * 4, dtype=torch.float64, device="cuda")
    rc = L.mf_refine_triggers_static(seg.handle, None, ctypes.c_void_p(th.data_ptr()), n, None,
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(out.data_ptr() + 8 * n), None)
    assert rc == mf._native.MF_EINVAL
    assert b"4096" in L.mf_last_error()
