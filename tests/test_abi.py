"""The C-ABI library builds, loads and exports every entry point that
include/mfgb.h declares; argument errors come back as MF_EINVAL without any
device work (these run without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_0906_4175_gb300 import build, _native
    build.build()
    return _native.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "mfgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mf_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("mf_bank_create", "mf_segment_upload", "mf_filter_bank", "mf_refine_triggers"):
        assert n in names


def test_every_declared_symbol_is_exported(L):
    from paper_0906_4175_gb300 import _native
    for name in _declared():
        assert hasattr(L, name), name
        assert name in _native.SIGNATURES, name


def test_version(L):
    assert b"sm_103a" in L.mf_version()


def test_invalid_arguments_without_device(L):
    from paper_0906_4175_gb300 import _native
    EINVAL = _native.MF_EINVAL
    h = ctypes.c_void_p()
    m = np.array([1.4, -1.0])
    assert L.mf_bank_create(m.ctypes.data, m.ctypes.data, 0, None, ctypes.byref(h)) == EINVAL
    assert L.mf_bank_create(m.ctypes.data, m.ctypes.data, 2, None, None) == EINVAL
    assert b"NULL" in L.mf_last_error()
    s = np.zeros(1000, dtype=np.float32)
    assert L.mf_segment_upload(s.ctypes.data, 1000, 4096.0, None, 150.0, 1.0, 0, None, ctypes.byref(h)) == EINVAL
    assert b"power of two" in L.mf_last_error()
    assert L.mf_segment_upload(s.ctypes.data, 1 << 23, 4096.0, None, 150.0, 1.0, 0, None, ctypes.byref(h)) == EINVAL
    assert L.mf_segment_upload(s.ctypes.data, 1024, -1.0, None, 150.0, 1.0, 0, None, ctypes.byref(h)) == EINVAL
    assert L.mf_filter_bank(None, None, 0, 6.0, None, None, 0, None, None) == EINVAL
    assert L.mf_refine_triggers(None, None, None, 1, None, None, None, None) == EINVAL
    g = np.zeros(2, dtype=np.float64)
    assert L.mf_synth_segment(g.ctypes.data, 100, 4096.0, 40.0, None, 150.0, 1.0, None, 0, 1.0,
                              g.ctypes.data, None) == EINVAL
    p = _native.BankParams(40.0, 3, 0, 0, 0)
    assert L.mf_bank_create(m.ctypes.data, m.ctypes.data, 2, ctypes.byref(p), ctypes.byref(h)) == _native.MF_ENOTSUP
    p = _native.BankParams(40.0, 4, 0, 0, 3)   # fft_mode past MF_FFT_TC_BF16
    assert L.mf_bank_create(m.ctypes.data, m.ctypes.data, 2, ctypes.byref(p), ctypes.byref(h)) == _native.MF_ENOTSUP
    assert b"fft_mode" in L.mf_last_error()
    assert L.mf_bank_destroy(None) == 0 and L.mf_segment_destroy(None) == 0


def test_invalid_arguments_of_the_later_entry_points(L):
    """chi^2, events, batched FFT, multi-row refinement and segment refresh
    reject bad arguments before any device work."""
    from paper_0906_4175_gb300 import _native
    EINVAL = _native.MF_EINVAL
    x = np.zeros(8, dtype=np.float32)
    n = np.zeros(1, dtype=np.int64)
    # mf_chisq_series: NULL bank / segment / outputs
    assert L.mf_chisq_series(None, None, None, 1, 16, None, None, None) == EINVAL
    # mf_chisq_points: NULL bank, bad stride
    assert L.mf_chisq_points(None, None, 1, None, 6, 1, 16, None, None) == EINVAL
    # mf_cluster_triggers: NULLs, negative window, bad capacity
    assert L.mf_cluster_triggers(None, None, 16, 4, 1, 1024, 8, None, 16, None, None) == EINVAL
    assert L.mf_cluster_triggers(x.ctypes.data, n.ctypes.data, 16, 4, 1, 1024, -1, x.ctypes.data, 16,
                                 n.ctypes.data, None) == EINVAL
    assert L.mf_cluster_triggers(x.ctypes.data, n.ctypes.data, 0, 4, 1, 1024, 8, x.ctypes.data, 16,
                                 n.ctypes.data, None) == EINVAL
    # mf_fft_c2c: length, sign, alignment
    assert L.mf_fft_c2c(x.ctypes.data, x.ctypes.data, 1000, 1, -1, None) == EINVAL
    assert b"power of two" in L.mf_last_error()
    assert L.mf_fft_c2c(x.ctypes.data, x.ctypes.data, 1024, 1, 2, None) == EINVAL
    assert L.mf_fft_c2c(x.ctypes.data + 4, x.ctypes.data, 1024, 1, 1, None) == EINVAL
    assert L.mf_fft_c2c(x.ctypes.data, x.ctypes.data, 1024, 0, 1, None) == EINVAL
    # mf_refine_triggers_multi: NULL row map, too many segments
    assert L.mf_refine_triggers_multi(None, 1, None, None, None, 1, None, None, None, None) == EINVAL
    assert L.mf_refine_triggers_multi(x.ctypes.data, 257, x.ctypes.data, None, x.ctypes.data, 1, None,
                                      x.ctypes.data, x.ctypes.data, None) == EINVAL
    # mf_segment_refresh: NULL segment
    assert L.mf_segment_refresh(None, x.ctypes.data, 1, None) == EINVAL


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    """No CPU fallback: a missing library is an ImportError, not a silent substitute."""
    from paper_0906_4175_gb300 import _native
    monkeypatch.setattr(_native, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_native, "_lib", None)
    with pytest.raises(ImportError):
        _native.lib()


def test_product_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_0906_4175_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "mf_oracle" not in txt, f
