"""Template sharding (the multi-device split of a bank by template range), its
host logic on CPU: the cost-balanced partition, the merge of per-shard
outputs, and the gather over world_size-2 gloo ranks.  The per-shard outputs
here come from the FP64 oracle run on each shard's templates, so the merged
result can be compared with the oracle's whole-bank result."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sh():
    from paper_0906_4175_gb300 import build
    build.build()
    from paper_0906_4175_gb300 import shard
    oracle.build()
    return shard


def _costs(m1, m2, shapes, f_low=40.0):
    """The modelled per-template cost, recomputed from the oracle's band rule."""
    c = np.zeros(m1.size)
    for i, (a, b) in enumerate(zip(m1, m2)):
        for N, fs in shapes:
            lo, hi = oracle.band(N, fs, f_low, oracle.f_isco(a, b))
            c[i] += 16.0 * N + 8.0 * max(0, hi - lo)
    return c


@pytest.mark.parametrize("parts", [1, 2, 3, 8])
def test_partition_is_contiguous_and_balanced(sh, parts):
    rng = np.random.default_rng(parts)
    m1 = rng.uniform(1.0, 20.0, 200)
    m2 = rng.uniform(1.0, 15.0, 200)
    shapes = [(1 << 16, 4096.0), (1 << 14, 2048.0)]
    st = sh.partition(m1, m2, shapes, parts)
    assert st[0] == 0 and st[-1] == m1.size and np.all(np.diff(st) > 0)
    c = _costs(m1, m2, shapes)
    load = np.array([c[st[r]:st[r + 1]].sum() for r in range(parts)])
    # each cut is the template boundary nearest to its quantile of the cost
    assert load.max() <= c.sum() / parts + c.max()
    assert load.min() >= c.sum() / parts - c.max()


def test_partition_rejects_bad_arguments(sh):
    from paper_0906_4175_gb300 import MFError
    with pytest.raises(MFError):
        sh.partition([1.4, 1.4], [1.4, 1.4], [(1 << 12, 4096.0)], 3)   # more parts than templates
    with pytest.raises(MFError):
        sh.partition([1.4, -1.0], [1.4, 1.4], [(1 << 12, 4096.0)], 1)


def _oracle_shard(m1, m2, s64, fs, thr, first, last, n_seg=1):
    """One shard's outputs in the product's record layout, template indices bank-wide."""
    from paper_0906_4175_gb300 import PEAK_DTYPE, TRIG_DTYPE
    pk, tr, n, _ = oracle.filter_bank(m1[first:last], m2[first:last], s64, fs, 40.0, thr)
    p = np.zeros(pk.size, dtype=PEAK_DTYPE)
    for f in ("rho", "j", "z_re", "z_im"):
        p[f] = pk[f]
    t = np.zeros(tr.size, dtype=TRIG_DTYPE)
    for f in ("tmpl", "seg", "j", "rho", "z_re", "z_im"):
        t[f] = tr[f]
    t["tmpl"] += first
    return p, t, n


def _tiny_bank():
    wl = workloads.small(seed=4, N=1 << 12, fs=2048.0, n_templates=7, m_lo=1.1, m_hi=3.0, snr=15.0)
    spec = wl.segments[0]
    s64 = oracle.synth(spec.normals(), spec.N, spec.fs, wl.f_low, spec.injections).astype(np.float32).astype(
        np.float64)
    return wl, spec, s64


def test_merge_of_shards_equals_whole_bank(sh):
    wl, spec, s64 = _tiny_bank()
    st = sh.partition(wl.m1, wl.m2, [(spec.N, spec.fs)], 3)
    shards = [_oracle_shard(wl.m1, wl.m2, s64, spec.fs, 3.0, st[r], st[r + 1]) for r in range(3)]
    peaks, trig, n = sh.merge(shards)
    whole = _oracle_shard(wl.m1, wl.m2, s64, spec.fs, 3.0, 0, wl.n_templates)
    assert n == whole[2] and trig.size == n
    assert np.array_equal(peaks, whole[0])
    assert np.array_equal(trig, whole[1])
    keys = list(zip(trig["tmpl"], trig["seg"], trig["j"]))
    assert keys == sorted(keys)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_0906_4175_gb300 import shard
    import test_shard as T
    wl, spec, s64 = T._tiny_bank()
    st = shard.partition(wl.m1, wl.m2, [(spec.N, spec.fs)], world)
    local = T._oracle_shard(wl.m1, wl.m2, s64, spec.fs, 3.0, st[rank], st[rank + 1])
    peaks, trig, n = shard.gather(local)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, peaks.tobytes(), trig.tobytes(), n))


@pytest.mark.timeout(180)
def test_gather_over_two_gloo_ranks(sh):
    pytest.importorskip("torch")
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=150) for _ in ps)
    for p in ps:
        p.join(timeout=30)
        assert p.exitcode == 0
    wl, spec, s64 = _tiny_bank()
    whole = _oracle_shard(wl.m1, wl.m2, s64, spec.fs, 3.0, 0, wl.n_templates)
    for _, pb, tb, n in res:      # every rank holds the merged bank result
        assert pb == whole[0].tobytes() and tb == whole[1].tobytes() and n == whole[2]
