"""GB300-native frequency-domain matched filter of arXiv:0906.4175.

For each template (m1, m2) of a bank and each data segment the library forms
Eq. (1)  z(t) = 4 int h~_c(f) s~*(f)/S_n(f) e^{2 pi i f t} df  with the 2PN
stationary-phase template (Sec. 1.1), Eq. (3) rho = |z|/sigma with Eq. (4)
sigma^2 = 4 int |h~_c|^2/S_n df, the per-segment argmax and every sample
above threshold -- all in hand-written sm_103a CUDA behind the C ABI of
include/mfgb.h.  This module only marshals arguments: PyTorch supplies device
memory and streams.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from ._native import (EVENT_DTYPE, INJ_DTYPE, MF_EINVAL, MF_EOVERFLOW, MF_ETIMEOUT, MF_FFT_FP32, MF_FFT_TC_BF16,
                      MF_FFT_TC_FP16, MF_OK, MF_PHASE_ANCHOR,
                      MF_PHASE_FP32, MF_PHASE_FP64, PEAK_DTYPE, TRIG_DTYPE, BankParams, MFError, check)

__all__ = ["Bank", "Segment", "filter_bank", "chisq_series", "chisq_points", "cluster_triggers",
           "events_to_numpy", "EVENT_DTYPE", "fft", "autotune", "synth_segment", "refine", "RefineFn", "MFError",
           "PEAK_DTYPE", "TRIG_DTYPE", "INJ_DTYPE", "MF_PHASE_ANCHOR", "MF_PHASE_FP64", "MF_PHASE_FP32",
           "MF_FFT_FP32", "MF_FFT_TC_FP16", "MF_FFT_TC_BF16",
           "peaks_to_numpy", "triggers_to_numpy", "version"]


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def version() -> str:
    return _native.lib().mf_version().decode()


def params(f_low: float = 40.0, phase_mode: int = MF_PHASE_ANCHOR, pn_order: int = 4,
           amp_order: int = 0, fft_mode: int = MF_FFT_FP32) -> BankParams:
    return BankParams(f_low, pn_order, amp_order, phase_mode, fft_mode)


class Bank:
    """mf_bank_create: template constants for masses m1, m2 (solar masses).

    With ``first``/``count`` the bank holds templates [first, first + count) of
    the mass list (mf_bank_create_shard: a shard of a bank split by template
    range, numbered 0 .. count-1, filtered as the whole list's bank would)."""

    def __init__(self, m1, m2, f_low: float = 40.0, phase_mode: int = MF_PHASE_ANCHOR, fft_mode: int = MF_FFT_FP32,
                 first: int = 0, count: int = None):
        m1 = np.ascontiguousarray(m1, dtype=np.float64)
        m2 = np.ascontiguousarray(m2, dtype=np.float64)
        if m1.shape != m2.shape or m1.ndim != 1:
            raise ValueError("m1 and m2 must be 1-D arrays of the same length")
        self.params = params(f_low, phase_mode, fft_mode=fft_mode)
        h = ctypes.c_void_p()
        L = _native.lib()
        if count is None and first == 0:
            check(L.mf_bank_create(m1.ctypes.data, m2.ctypes.data, m1.size, ctypes.byref(self.params),
                                   ctypes.byref(h)))
            count = m1.size
        else:
            count = m1.size - first if count is None else count
            check(L.mf_bank_create_shard(m1.ctypes.data, m2.ctypes.data, m1.size, ctypes.byref(self.params),
                                         int(first), int(count), ctypes.byref(h)))
        self._h = h
        self.n = int(count)
        self.first = int(first)
        self.m1, self.m2 = m1[first:first + count], m2[first:first + count]

    @property
    def handle(self):
        return self._h

    def check(self, stream=None, allow_timeout: bool = False) -> int:
        """mf_bank_check: sync and return MF_OK / MF_EOVERFLOW (raises on timeout unless allowed)."""
        allow = (MF_EOVERFLOW, MF_ETIMEOUT) if allow_timeout else (MF_EOVERFLOW,)
        return check(_native.lib().mf_bank_check(self._h, _stream_ptr(stream)), allow=allow)

    def debug_stall(self, unit: int, spin_limit: int = 0):
        """Test hook (mf_bank_debug_stall): make a unit's bounded wait run out."""
        check(_native.lib().mf_bank_debug_stall(self._h, int(unit), int(spin_limit)))

    def profile(self, on: bool = True):
        """Record per-kernel CUDA events in later filter_bank calls (mf_bank_profile)."""
        check(_native.lib().mf_bank_profile(self._h, 1 if on else 0))

    def profile_read(self):
        """{stage: (ms, algorithmic bytes, launches)} since the last read."""
        ns = len(_native.STAGES)
        ms = (ctypes.c_double * ns)()
        by = (ctypes.c_double * ns)()
        nl = (ctypes.c_int64 * ns)()
        check(_native.lib().mf_bank_profile_read(self._h, ms, by, nl))
        return {name: (ms[i], by[i], nl[i]) for i, name in enumerate(_native.STAGES)}

    def close(self):
        if getattr(self, "_h", None):
            _native.lib().mf_bank_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    """Kernels launched by libmfgb in this process so far."""
    n = ctypes.c_int64()
    check(_native.lib().mf_launch_count(ctypes.byref(n)))
    return int(n.value)


class Segment:
    """mf_segment_upload: s (torch float32 tensor on cuda, or numpy float32 on host)."""

    def __init__(self, s, fs: float, psd=None, psd_f0: float = 150.0, psd_S0: float = 1.0, stream=None):
        torch = _torch()
        on_dev = isinstance(s, torch.Tensor) and s.is_cuda
        if on_dev:
            if s.dtype != torch.float32 or not s.is_contiguous():
                raise ValueError("device s must be a contiguous float32 tensor")
            ptr, N, keep = s.data_ptr(), s.numel(), s
        else:
            keep = np.ascontiguousarray(s, dtype=np.float32)
            ptr, N = keep.ctypes.data, keep.size
        psd_a = None if psd is None else np.ascontiguousarray(psd, dtype=np.float64)
        if psd_a is not None and psd_a.size != N // 2 + 1:
            raise ValueError("psd must hold N/2+1 values")
        h = ctypes.c_void_p()
        check(_native.lib().mf_segment_upload(ptr, N, fs, None if psd_a is None else psd_a.ctypes.data,
                                              psd_f0, psd_S0, 1 if on_dev else 0, _stream_ptr(stream),
                                              ctypes.byref(h)))
        self._h = h
        self._keep = keep
        self.N = int(N)
        self.fs = float(fs)

    @property
    def handle(self):
        return self._h

    def set_conditioning(self, mode: str):
        """mf_segment_set_conditioning: 'fp64' (default) or 'fp32' forward FFT
        in later refresh() calls."""
        m = {"fp64": _native.MF_COND_FP64, "fp32": _native.MF_COND_FP32}[mode]
        check(_native.lib().mf_segment_set_conditioning(self._h, m))

    def refresh(self, s, stream=None):
        """mf_segment_refresh: condition new samples (same N, fs and PSD) into
        this segment's device memory; capturable in a CUDA graph for device s
        after the first call."""
        torch = _torch()
        on_dev = isinstance(s, torch.Tensor) and s.is_cuda
        if on_dev:
            if s.dtype != torch.float32 or not s.is_contiguous() or s.numel() != self.N:
                raise ValueError("device s must be a contiguous float32 tensor of N samples")
            ptr, keep = s.data_ptr(), s
        else:
            keep = np.ascontiguousarray(s, dtype=np.float32)
            if keep.size != self.N:
                raise ValueError("s must hold N samples")
            ptr = keep.ctypes.data
        check(_native.lib().mf_segment_refresh(self._h, ptr, 1 if on_dev else 0, _stream_ptr(stream)))
        self._keep = keep
        return self

    def close(self):
        if getattr(self, "_h", None):
            _native.lib().mf_segment_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def filter_bank(bank: Bank, segments, threshold: float, trig_cap: int = 1 << 20, stream=None,
                out=None):
    """mf_filter_bank over all (template, segment) pairs.

    Returns (peaks, triggers, n_trig) as torch device tensors:
    peaks  int32/float32 [n_templates * n_seg, 4] laid out as PEAK_DTYPE,
    triggers [trig_cap, 6] laid out as TRIG_DTYPE, n_trig int64 [1] (true count).
    ``out`` may pass preallocated (peaks, triggers, n_trig) tensors."""
    torch = _torch()
    segs = list(segments) if isinstance(segments, (list, tuple)) else [segments]
    arr = (ctypes.c_void_p * len(segs))(*[s.handle.value for s in segs])
    dev = torch.device("cuda", torch.cuda.current_device())
    if out is None:
        peaks = torch.empty((bank.n * len(segs), 4), dtype=torch.float32, device=dev)
        trig = torch.empty((max(trig_cap, 1), 6), dtype=torch.float32, device=dev)
        n_trig = torch.zeros(1, dtype=torch.int64, device=dev)
    else:
        peaks, trig, n_trig = out
    check(_native.lib().mf_filter_bank(bank.handle, arr, len(segs), float(threshold), peaks.data_ptr(),
                                       trig.data_ptr(), int(trig_cap), n_trig.data_ptr(),
                                       _stream_ptr(stream)))
    return peaks, trig, n_trig


def fft(x, sign: int = -1, out=None, stream=None):
    """mf_fft_c2c: batched complex FFT over the last axis of a complex64 cuda
    tensor (unnormalised; sign -1 forward, +1 inverse)."""
    torch = _torch()
    if x.dtype != torch.complex64 or not x.is_cuda or not x.is_contiguous():
        raise ValueError("x must be a contiguous complex64 cuda tensor")
    N = int(x.shape[-1])
    batch = int(x.numel() // N) if N else 0
    y = torch.empty_like(x) if out is None else out
    check(_native.lib().mf_fft_c2c(x.data_ptr(), y.data_ptr(), N, batch, int(sign), _stream_ptr(stream)))
    return y


def cluster_triggers(trig, n_trig, n_tmpl: int, n_seg: int, max_N: int, window: int, ev_cap: int = None,
                     stream=None):
    """mf_cluster_triggers: events from (tmpl, seg, j)-sorted triggers (the
    filter_bank outputs).  Returns (events float32 cuda [ev_cap, 8] laid out
    as EVENT_DTYPE, n_events int64 cuda [1], the true count)."""
    torch = _torch()
    dev = trig.device
    cap = int(trig.shape[0])
    ev_cap = cap if ev_cap is None else int(ev_cap)
    ev = torch.empty((max(ev_cap, 1), 8), dtype=torch.float32, device=dev)
    n_ev = torch.zeros(1, dtype=torch.int64, device=dev)
    check(_native.lib().mf_cluster_triggers(trig.data_ptr(), n_trig.data_ptr(), cap, int(n_tmpl), int(n_seg),
                                            int(max_N), int(window), ev.data_ptr(), ev_cap, n_ev.data_ptr(),
                                            _stream_ptr(stream)))
    return ev, n_ev


def events_to_numpy(ev, n_ev) -> np.ndarray:
    n = int(n_ev.item()) if hasattr(n_ev, "item") else int(n_ev)
    n = min(n, ev.shape[0])
    return ev[:n].detach().cpu().contiguous().numpy().view(EVENT_DTYPE).reshape(-1)


def chisq_points(bank: Bank, segments, rows, p: int = 16, stream=None):
    """mf_chisq_points: Eq. (5) chi^2 at the (tmpl, seg, j) of each row of a
    trigger [n, 6] or event [n, 8] tensor (cuda, 4-byte fields)."""
    torch = _torch()
    segs = list(segments) if isinstance(segments, (list, tuple)) else [segments]
    arr = (ctypes.c_void_p * len(segs))(*[sg.handle.value for sg in segs])
    if not rows.is_cuda or rows.dim() != 2 or rows.element_size() != 4 or not rows.is_contiguous():
        raise ValueError("rows must be a contiguous 2-D cuda tensor of 4-byte fields")
    n = int(rows.shape[0])
    out = torch.empty(max(n, 1), dtype=torch.float32, device=rows.device)
    check(_native.lib().mf_chisq_points(bank.handle, arr, len(segs), rows.data_ptr(), int(rows.shape[1]), n, int(p),
                                        out.data_ptr(), _stream_ptr(stream)))
    return out[:n]


def chisq_series(bank: Bank, segment: Segment, tmpl, p: int = 16, stream=None):
    """mf_chisq_series: Eq. (5) chi^2 at every sample for the bank templates
    tmpl (sequence of indices or an int32 cuda tensor).  Returns (chisq
    float32 cuda [n, N], edges int64 cuda [n, p+1])."""
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    t = tmpl if isinstance(tmpl, torch.Tensor) else torch.tensor(np.asarray(tmpl, dtype=np.int32), device=dev)
    t = t.to(device=dev, dtype=torch.int32).contiguous()
    n = int(t.numel())
    chisq = torch.empty((n, segment.N), dtype=torch.float32, device=dev)
    edges = torch.empty((n, p + 1), dtype=torch.int64, device=dev)
    check(_native.lib().mf_chisq_series(bank.handle, segment.handle, t.data_ptr(), n, int(p), chisq.data_ptr(),
                                        edges.data_ptr(), _stream_ptr(stream)))
    return chisq, edges


def autotune(bank: Bank, segments, threshold: float, repeats: int = 2, cache_path: str = None, stream=None):
    """mf_autotune: time the candidate schedules on this bank and keep the fastest."""
    segs = list(segments) if isinstance(segments, (list, tuple)) else [segments]
    arr = (ctypes.c_void_p * len(segs))(*[s.handle.value for s in segs])
    check(_native.lib().mf_autotune(bank.handle, arr, len(segs), float(threshold), int(repeats),
                                    cache_path.encode() if cache_path else None, _stream_ptr(stream)))


def peaks_to_numpy(peaks) -> np.ndarray:
    a = peaks.detach().cpu().contiguous().numpy()
    return a.view(PEAK_DTYPE).reshape(-1)


def triggers_to_numpy(trig, n_trig) -> np.ndarray:
    n = int(n_trig.item()) if hasattr(n_trig, "item") else int(n_trig)
    n = min(n, trig.shape[0])
    a = trig[:n].detach().cpu().contiguous().numpy()
    return a.view(TRIG_DTYPE).reshape(-1)


def synth_segment(g, N: int, fs: float, f_low: float = 40.0, injections=None, psd=None,
                  psd_f0: float = 150.0, psd_S0: float = 1.0, noise_scale: float = 1.0, stream=None):
    """mf_synth_segment: coloured Gaussian noise + injections -> float32 cuda tensor [N].
    g: 2*(N/2) standard normals (numpy or cuda float64 tensor)."""
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    gt = g if isinstance(g, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(g, dtype=np.float64))
    gt = gt.to(device=dev, dtype=torch.float64).contiguous()
    if gt.numel() != 2 * (N // 2):
        raise ValueError("g must hold 2*(N/2) normals")
    inj = np.zeros(0, dtype=INJ_DTYPE) if injections is None else np.ascontiguousarray(injections, dtype=INJ_DTYPE)
    psd_a = None if psd is None else np.ascontiguousarray(psd, dtype=np.float64)
    s = torch.empty(N, dtype=torch.float32, device=dev)
    check(_native.lib().mf_synth_segment(gt.data_ptr(), N, fs, f_low,
                                         None if psd_a is None else psd_a.ctypes.data, psd_f0, psd_S0,
                                         inj.ctypes.data if inj.size else None, inj.size, noise_scale,
                                         s.data_ptr(), _stream_ptr(stream)))
    return s


def _refine_args(theta, band, torch):
    theta = theta.contiguous()
    if theta.dtype != torch.float64 or not theta.is_cuda or theta.dim() != 2 or theta.shape[1] != 3:
        raise ValueError("theta must be a float64 cuda tensor of shape [n, 3]")
    n = theta.shape[0]
    bp = None
    if band is not None:
        band = band.contiguous()
        if band.dtype != torch.int64 or not band.is_cuda or tuple(band.shape) != (n, 2):
            raise ValueError("band must be an int64 cuda tensor of shape [n, 2]")
        bp = band.data_ptr()
    obj = torch.empty(n, dtype=torch.float64, device=theta.device)
    grad = torch.empty((n, 3), dtype=torch.float64, device=theta.device)
    return theta, n, bp, band, obj, grad


def refine(segment, theta, band=None, f_low: float = 40.0, stream=None,
           phase_mode: int = MF_PHASE_ANCHOR, row_seg=None):
    """mf_refine_triggers: rho^2 and d rho^2 / d(m1, m2, t) for theta [n, 3] (float64 cuda).

    segment: one Segment, or a list of Segments with row_seg (int32 cuda [n])
    naming each row's segment (mf_refine_triggers_multi, one launch).
    phase_mode: MF_PHASE_ANCHOR (FP64 anchors + FP32 Taylor, default) or
    MF_PHASE_FP64 (FP64 phase at every bin)."""
    torch = _torch()
    theta, n, bp, band, obj, grad = _refine_args(theta, band, torch)
    p = params(f_low, phase_mode=phase_mode)
    if isinstance(segment, (list, tuple)):
        if row_seg is None:
            raise ValueError("row_seg is required with a list of segments")
        row_seg = row_seg.contiguous()
        if row_seg.dtype != torch.int32 or not row_seg.is_cuda or row_seg.numel() != n:
            raise ValueError("row_seg must be an int32 cuda tensor of n entries")
        arr = (ctypes.c_void_p * len(segment))(*[s.handle.value for s in segment])
        check(_native.lib().mf_refine_triggers_multi(arr, len(segment), row_seg.data_ptr(), ctypes.byref(p),
                                                     theta.data_ptr(), n, bp, obj.data_ptr(), grad.data_ptr(),
                                                     _stream_ptr(stream)))
    else:
        check(_native.lib().mf_refine_triggers(segment.handle, ctypes.byref(p), theta.data_ptr(), n, bp,
                                               obj.data_ptr(), grad.data_ptr(), _stream_ptr(stream)))
    return obj, grad


def _make_refine_fn():
    torch = _torch()

    class RefineFn(torch.autograd.Function):
        """rho^2(m1, m2, t) of each trigger row with the hand-written adjoint.

        forward(theta [n, 3] float64 cuda, segment, band=None, f_low=40, row_seg=None)
        -> rho^2 [n]; segment may be a list of Segments with row_seg (int32
        cuda [n]).  backward returns grad_out[:, None] * d rho^2 / d theta (no
        gradient for segment, band, f_low, row_seg)."""

        @staticmethod
        def forward(ctx, theta, segment, band=None, f_low=40.0, row_seg=None):
            obj, grad = refine(segment, theta.detach(), band=band, f_low=f_low, row_seg=row_seg)
            ctx.save_for_backward(grad)
            return obj

        @staticmethod
        def backward(ctx, grad_out):
            (grad,) = ctx.saved_tensors
            return grad_out[:, None] * grad, None, None, None, None

    return RefineFn


class _LazyRefineFn:
    _cls = None

    def __getattr__(self, name):
        if _LazyRefineFn._cls is None:
            _LazyRefineFn._cls = _make_refine_fn()
        return getattr(_LazyRefineFn._cls, name)


RefineFn = _LazyRefineFn()
