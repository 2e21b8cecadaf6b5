"""Plain FP64 CPU oracle for the matched filter of arXiv:0906.4175 (Eqs. 1-4).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA path
(``paper_0906_4175_gb300``) never imports it, and the two share no code.

The arithmetic lives in ``mf_oracle.c`` (plain C, FP64, its own radix-2 FFT);
this module only compiles it with gcc and marshals numpy arrays through
ctypes.  Each wrapper names the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmforacle.so")
_lock = threading.Lock()
_lib = None

MSUN_S = 4.925490947e-6  # G Msun / c^3 [s], the value the C oracle uses


def build(force: bool = False) -> str:
    """Compile mf_oracle.c into oracle/_build/libmforacle.so (gcc, -O2, OpenMP).

    -ffp-contract=off keeps the FP64 arithmetic identical on x86 and Arm.
    """
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Peak(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("j", ctypes.c_int64),
                ("z_re", ctypes.c_double), ("z_im", ctypes.c_double),
                ("sigma", ctypes.c_double), ("k_lo", ctypes.c_int64),
                ("k_hi", ctypes.c_int64)]


class Trigger(ctypes.Structure):
    _fields_ = [("tmpl", ctypes.c_int32), ("seg", ctypes.c_int32),
                ("j", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("rho", ctypes.c_double), ("z_re", ctypes.c_double),
                ("z_im", ctypes.c_double)]


class Injection(ctypes.Structure):
    _fields_ = [("m1", ctypes.c_double), ("m2", ctypes.c_double),
                ("snr", ctypes.c_double), ("j0", ctypes.c_int64),
                ("phi", ctypes.c_double)]


PEAK_DTYPE = np.dtype([("rho", "f8"), ("j", "i8"), ("z_re", "f8"), ("z_im", "f8"),
                       ("sigma", "f8"), ("k_lo", "i8"), ("k_hi", "i8")])
TRIG_DTYPE = np.dtype([("tmpl", "i4"), ("seg", "i4"), ("j", "i4"), ("pad", "i4"),
                       ("rho", "f8"), ("z_re", "f8"), ("z_im", "f8")])
INJ_DTYPE = np.dtype([("m1", "f8"), ("m2", "f8"), ("snr", "f8"), ("j0", "i8"), ("phi", "f8")])

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.c_int64
_P = ctypes.c_void_p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.or_fft.argtypes = [_P, _P, _I64, ctypes.c_int]
            L.or_fft.restype = ctypes.c_int
            L.or_psd_eq2.argtypes = [ctypes.c_double] * 3
            L.or_psd_eq2.restype = ctypes.c_double
            L.or_psi.argtypes = [ctypes.c_double] * 3
            L.or_psi.restype = ctypes.c_double
            L.or_band.argtypes = [_I64, ctypes.c_double, ctypes.c_double, ctypes.c_double, _P, _P]
            L.or_htilde.argtypes = [ctypes.c_double, ctypes.c_double, _I64, ctypes.c_double,
                                    ctypes.c_double, _P, _P, _P, _P]
            L.or_psd_bins.argtypes = [_I64, ctypes.c_double, ctypes.c_double, ctypes.c_double, _P]
            L.or_data_spectrum.argtypes = [_P, _I64, ctypes.c_double, _P, _P]
            L.or_data_spectrum.restype = ctypes.c_int
            L.or_filter_template.argtypes = [ctypes.c_double, ctypes.c_double, _P, _P, _P, _I64,
                                             ctypes.c_double, ctypes.c_double, _P, _P, _P, _P,
                                             _P, _P]
            L.or_filter_template.restype = ctypes.c_int
            L.or_filter_bank.argtypes = [_P, _P, _I64, _P, _I64, ctypes.c_double, ctypes.c_double,
                                         _P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, _P, _P, _I64, _P, ctypes.c_int]
            L.or_filter_bank.restype = ctypes.c_int
            L.or_synth.argtypes = [_P, _I64, ctypes.c_double, ctypes.c_double, _P, ctypes.c_double,
                                   ctypes.c_double, _P, _I64, ctypes.c_double, _P]
            L.or_synth.restype = ctypes.c_int
            L.or_refine_objective.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              _P, _P, _P, _I64, ctypes.c_double, _I64, _I64, _P]
            L.or_refine_objective.restype = ctypes.c_double
            L.or_refine.argtypes = [_P, _I64, _P, _I64, ctypes.c_double, ctypes.c_double, _P,
                                    ctypes.c_double, ctypes.c_double, _P, _P, _P]
            L.or_refine.restype = ctypes.c_int
            L.or_chisq_series.argtypes = [ctypes.c_double, ctypes.c_double, _P, _P, _P, _I64, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, _P, _P, _P, _P, _P]
            L.or_chisq_series.restype = ctypes.c_int
            L.or_cluster.argtypes = [_P, _I64, ctypes.c_int32, _P, _I64]
            L.or_cluster.restype = ctypes.c_int64
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Wrappers.  Arrays are numpy float64 unless stated.
# --------------------------------------------------------------------------

def fft(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised radix-2 DFT  X_k = sum_n x_n exp(sign 2 pi i n k / N)."""
    x = np.asarray(x, dtype=np.complex128)
    re = np.ascontiguousarray(x.real.copy())
    im = np.ascontiguousarray(x.imag.copy())
    rc = lib().or_fft(_ptr(re), _ptr(im), re.size, int(sign))
    if rc != 0:
        raise ValueError("or_fft: length must be a power of two")
    return re + 1j * im


def psd_eq2(f, f0: float = 150.0, S0: float = 1.0):
    """Eq. (2): initial-LIGO PSD at frequency f (scalar or array)."""
    L = lib()
    f = np.asarray(f, dtype=np.float64)
    out = np.array([L.or_psd_eq2(float(v), f0, S0) for v in f.ravel()])
    return out.reshape(f.shape) if f.ndim else float(out[0])


def psd_bins(N: int, fs: float, f0: float = 150.0, S0: float = 1.0) -> np.ndarray:
    """Eq. (2) on bins k = 0..N/2 (S[0] = inf)."""
    S = np.empty(N // 2 + 1)
    lib().or_psd_bins(N, fs, f0, S0, _ptr(S))
    return S


def psi(m1: float, m2: float, f) -> np.ndarray:
    """2PN stationary-phase phase Psi(f) with t_c = phi_c = 0 (Sec. 1.1 templates)."""
    L = lib()
    f = np.asarray(f, dtype=np.float64)
    out = np.array([L.or_psi(m1, m2, float(v)) for v in f.ravel()])
    return out.reshape(f.shape) if f.ndim else float(out[0])


def band(N: int, fs: float, f_low: float, f_cut: float):
    """Band rule of Sec. 1.1 -> (k_lo, k_hi), half-open."""
    lo = ctypes.c_int64()
    hi = ctypes.c_int64()
    lib().or_band(N, fs, f_low, f_cut, ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def f_isco(m1: float, m2: float) -> float:
    """1 / (6^(3/2) pi M), M in seconds (the same FP64 expression the C oracle uses)."""
    Ms = (m1 + m2) * MSUN_S
    return 1.0 / (6.0 * np.sqrt(6.0) * np.pi * Ms)


def htilde(m1: float, m2: float, N: int, fs: float, f_low: float):
    """h~_k on k = 0..N/2 (complex128) and its band (k_lo, k_hi)."""
    re = np.empty(N // 2 + 1)
    im = np.empty(N // 2 + 1)
    lo = ctypes.c_int64()
    hi = ctypes.c_int64()
    lib().or_htilde(m1, m2, N, fs, f_low, _ptr(re), _ptr(im), ctypes.byref(lo), ctypes.byref(hi))
    return re + 1j * im, (lo.value, hi.value)


def data_spectrum(s: np.ndarray, fs: float) -> np.ndarray:
    """s~_k = dt DFT(s)_k on k = 0..N/2."""
    s = _f64(s)
    N = s.size
    re = np.empty(N // 2 + 1)
    im = np.empty(N // 2 + 1)
    lib().or_data_spectrum(_ptr(s), N, fs, _ptr(re), _ptr(im))
    return re + 1j * im


def filter_template(m1, m2, st: np.ndarray, S: np.ndarray, N: int, fs: float, f_low: float):
    """Eqs. (1), (3), (4) for one template: returns dict(z, rho, sigma, k_lo, k_hi)."""
    st_re = _f64(st.real)
    st_im = _f64(st.imag)
    S = _f64(S)
    z_re = np.empty(N)
    z_im = np.empty(N)
    rho = np.empty(N)
    sigma = ctypes.c_double()
    lo = ctypes.c_int64()
    hi = ctypes.c_int64()
    rc = lib().or_filter_template(m1, m2, _ptr(st_re), _ptr(st_im), _ptr(S), N, fs, f_low,
                                  _ptr(z_re), _ptr(z_im), _ptr(rho), ctypes.byref(sigma),
                                  ctypes.byref(lo), ctypes.byref(hi))
    if rc != 0:
        raise RuntimeError("or_filter_template failed: %d" % rc)
    return dict(z=z_re + 1j * z_im, rho=rho, sigma=sigma.value, k_lo=lo.value, k_hi=hi.value)


def chisq_series(m1, m2, st: np.ndarray, S: np.ndarray, N: int, fs: float, f_low: float, p: int = 16,
                 edges=None):
    """Eq. (5) for one template: chi^2 at every sample with p equal-sigma^2
    sub-bands (Sec. 1.2).  edges: optional p+1 band edges replacing the
    equal-share rule.  Returns dict(chisq, rho, edges, sig2_l)."""
    st_re = _f64(st.real)
    st_im = _f64(st.imag)
    S = _f64(S)
    chisq = np.empty(N)
    rho = np.empty(N)
    e_out = np.empty(p + 1, dtype=np.int64)
    sig2_l = np.empty(p)
    e_in = None if edges is None else np.ascontiguousarray(edges, dtype=np.int64)
    if e_in is not None and e_in.size != p + 1:
        raise ValueError("edges must hold p+1 values")
    rc = lib().or_chisq_series(float(m1), float(m2), _ptr(st_re), _ptr(st_im), _ptr(S), N, fs, f_low, p,
                               _ptr(e_in), _ptr(chisq), _ptr(rho), _ptr(e_out), _ptr(sig2_l))
    if rc != 0:
        raise RuntimeError("or_chisq_series failed: %d" % rc)
    return dict(chisq=chisq, rho=rho, edges=e_out, sig2_l=sig2_l)


EVENT_DTYPE = np.dtype([("tmpl", "i4"), ("seg", "i4"), ("j", "i4"), ("n_trig", "i4"), ("n_tmpl", "i4"),
                        ("pad", "i4"), ("rho", "f8"), ("z_re", "f8"), ("z_im", "f8")])


def cluster(triggers, window: int) -> np.ndarray:
    """Two-stage single-linkage clustering of triggers sorted by (tmpl, seg, j):
    per (template, segment) with gaps <= window samples, then the clusters'
    loudest members across templates by (segment, j).  Returns EVENT_DTYPE
    records sorted by (seg, j)."""
    t = np.ascontiguousarray(triggers, dtype=TRIG_DTYPE)
    ev = np.zeros(max(t.size, 1), dtype=EVENT_DTYPE)
    ne = lib().or_cluster(_ptr(t), t.size, int(window), _ptr(ev), ev.size)
    if ne < 0:
        raise RuntimeError("or_cluster failed")
    return ev[:ne]


def filter_bank(m1, m2, s, fs: float, f_low: float, thr: float, psd=None,
                f0: float = 150.0, S0: float = 1.0, seg_id: int = 0,
                trig_cap: int = 1 << 20, n_threads: int = 0):
    """Bank filter: per-template peaks and all samples with rho > thr.

    Returns (peaks[n_t] PEAK_DTYPE, triggers[n] TRIG_DTYPE in (template, j)
    order, true trigger count, threads used)."""
    m1 = _f64(m1)
    m2 = _f64(m2)
    s = _f64(s)
    n_t = m1.size
    N = s.size
    peaks = np.zeros(n_t, dtype=PEAK_DTYPE)
    trig = np.zeros(max(trig_cap, 1), dtype=TRIG_DTYPE)
    n_trig = ctypes.c_int64()
    psd_a = None if psd is None else _f64(psd)
    used = lib().or_filter_bank(_ptr(m1), _ptr(m2), n_t, _ptr(s), N, fs, f_low, _ptr(psd_a),
                                f0, S0, thr, seg_id, _ptr(peaks), _ptr(trig), trig_cap,
                                ctypes.byref(n_trig), n_threads)
    if used < 0:
        raise RuntimeError("or_filter_bank failed: %d" % used)
    n = n_trig.value
    return peaks, trig[:min(n, trig_cap)], n, used


def synth(g, N: int, fs: float, f_low: float, injections=None, psd=None,
          f0: float = 150.0, S0: float = 1.0, noise_scale: float = 1.0) -> np.ndarray:
    """Seeded coloured Gaussian noise (Eq. 2 PSD) plus frequency-domain injections.

    g: 2*(N/2) standard normals; injections: structured array INJ_DTYPE."""
    g = _f64(g)
    if g.size != 2 * (N // 2):
        raise ValueError("g must hold 2*(N/2) normals")
    inj = np.zeros(0, dtype=INJ_DTYPE) if injections is None else np.ascontiguousarray(
        injections, dtype=INJ_DTYPE)
    psd_a = None if psd is None else _f64(psd)
    s = np.empty(N)
    rc = lib().or_synth(_ptr(g), N, fs, f_low, _ptr(psd_a), f0, S0,
                        _ptr(inj) if inj.size else None, inj.size, noise_scale, _ptr(s))
    if rc != 0:
        raise RuntimeError("or_synth failed: %d" % rc)
    return s


def refine_objective(m1, m2, tc, st, S, N, fs, k_lo, k_hi):
    """J = rho^2 at continuous t (direct Eq. 1 sum) and dJ/d(m1, m2, t)."""
    st_re = _f64(st.real)
    st_im = _f64(st.imag)
    S = _f64(S)
    grad = np.empty(3)
    J = lib().or_refine_objective(m1, m2, tc, _ptr(st_re), _ptr(st_im), _ptr(S), N, fs,
                                  k_lo, k_hi, _ptr(grad))
    return J, grad


def refine(theta, s, fs: float, f_low: float, psd=None, f0=150.0, S0=1.0, bands=None):
    """Objective and gradient for n triggers theta[n, 3] = (m1, m2, t[s])."""
    theta = _f64(theta).reshape(-1, 3)
    s = _f64(s)
    n = theta.shape[0]
    obj = np.empty(n)
    grad = np.empty((n, 3))
    b = None
    if bands is not None:
        b = np.ascontiguousarray(bands, dtype=np.int64).reshape(n, 2)
    psd_a = None if psd is None else _f64(psd)
    lib().or_refine(_ptr(theta), n, _ptr(s), s.size, fs, f_low, _ptr(psd_a), f0, S0,
                    _ptr(b), _ptr(obj), _ptr(grad))
    return obj, grad
