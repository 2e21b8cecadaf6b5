"""Template sharding of a bank (the paper's projection to several GPUs, Sec. 4).

Templates are independent (Sec. 2: data parallelism over templates and
segments), so a bank splits by template range: every shard filters the same
segments with its own templates and the results are merged.  Nothing of the
filter itself crosses a shard boundary; the only exchange is the merge of
the outputs:

* peaks are laid out template-major (template t, segment s at t * n_seg + s),
  so the shards' peaks concatenated in range order are the bank's peaks;
* triggers are sorted by (template, segment, j) within a shard and the ranges
  are disjoint and ascending, so the shards' triggers, with the shard's first
  template added to their template index, concatenated in range order are
  the bank's triggers in the same order.

``partition`` calls mf_bank_partition (cost-balanced contiguous ranges),
``shard_bank`` builds one shard (mf_bank_create_shard: the anchor spacing of
the whole list, so results are bit-identical to the whole bank), ``merge``
joins host copies of per-shard outputs, and ``gather`` collects them over a
torch.distributed process group (one process per device) on every rank.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import Bank, params, peaks_to_numpy, triggers_to_numpy
from . import _native
from ._native import MF_PHASE_ANCHOR, PEAK_DTYPE, TRIG_DTYPE, check


def partition(m1, m2, segment_shapes, parts: int, f_low: float = 40.0) -> np.ndarray:
    """mf_bank_partition: ``parts + 1`` range starts (int64) over the bank.
    segment_shapes: iterable of (N, fs) of the segments every shard filters."""
    m1 = np.ascontiguousarray(m1, dtype=np.float64)
    m2 = np.ascontiguousarray(m2, dtype=np.float64)
    shapes = list(segment_shapes)
    seg_N = np.ascontiguousarray([int(n) for n, _ in shapes], dtype=np.int64)
    seg_fs = np.ascontiguousarray([float(f) for _, f in shapes], dtype=np.float64)
    starts = np.zeros(int(parts) + 1, dtype=np.int64)
    p = params(f_low)
    check(_native.lib().mf_bank_partition(m1.ctypes.data, m2.ctypes.data, m1.size, ctypes.byref(p),
                                          seg_N.ctypes.data, seg_fs.ctypes.data, len(shapes), int(parts),
                                          starts.ctypes.data))
    return starts


def shard_bank(m1, m2, starts, rank: int, f_low: float = 40.0, phase_mode: int = MF_PHASE_ANCHOR) -> Bank:
    """The Bank of shard ``rank``: templates [starts[rank], starts[rank + 1])."""
    first, last = int(starts[rank]), int(starts[rank + 1])
    return Bank(m1, m2, f_low=f_low, phase_mode=phase_mode, first=first, count=last - first)


def local_results(bank: Bank, peaks, trig, n_trig):
    """Host copies of one shard's filter_bank outputs with bank-wide template
    indices: (peaks PEAK_DTYPE, triggers TRIG_DTYPE, true trigger count)."""
    p = peaks_to_numpy(peaks)
    t = triggers_to_numpy(trig, n_trig).copy()
    t["tmpl"] += bank.first
    return p, t, int(n_trig.item())


def merge(shards):
    """Join per-shard (peaks, triggers, n_trig) given in range order into the
    bank's (peaks, triggers, n_trig).  n_trig is the sum of the shards' true
    counts (a shard whose trigger buffer overflowed contributes what it kept)."""
    shards = list(shards)
    peaks = np.concatenate([np.asarray(p, dtype=PEAK_DTYPE) for p, _, _ in shards]) if shards else \
        np.zeros(0, dtype=PEAK_DTYPE)
    trig = np.concatenate([np.asarray(t, dtype=TRIG_DTYPE) for _, t, _ in shards]) if shards else \
        np.zeros(0, dtype=TRIG_DTYPE)
    return peaks, trig, int(sum(int(n) for _, _, n in shards))


def gather(local, group=None):
    """All ranks' ``local`` = (peaks, triggers, n_trig) host results, merged in
    rank order (rank r holding shard r), returned on every rank."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    out = [None] * world
    dist.all_gather_object(out, (np.asarray(local[0]).tobytes(), np.asarray(local[1]).tobytes(), int(local[2])),
                           group=group)
    shards = [(np.frombuffer(p, dtype=PEAK_DTYPE), np.frombuffer(t, dtype=TRIG_DTYPE), n) for p, t, n in out]
    return merge(shards)
