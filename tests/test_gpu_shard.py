"""Template sharding on the GPU: a bank split into cost-balanced template
ranges, each shard filtered on its own (here one after another on one
device), merges into exactly the whole bank's peaks and triggers."""
import numpy as np
import pytest

import workloads
from mfgb_testutil import oracle_segment

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_4175_gb300 import build
    build.build()
    import paper_0906_4175_gb300 as m
    return m


@pytest.mark.parametrize("N,parts", [(1 << 16, 3), (1 << 20, 4)])
def test_shards_merge_bit_identical_to_whole_bank(mf, N, parts):
    import torch
    from paper_0906_4175_gb300 import shard
    rng = np.random.default_rng(N + parts)
    m1 = rng.uniform(1.0, 6.0, 61)
    m2 = rng.uniform(1.0, 6.0, 61)
    spec = workloads.SegmentSpec(N, 4096.0, 40 + parts)
    s32, _ = oracle_segment(spec)
    seg = mf.Segment(torch.from_numpy(s32).cuda(), spec.fs)
    whole = mf.Bank(m1, m2)
    p, t, n = mf.filter_bank(whole, [seg], 5.0, trig_cap=1 << 18)
    assert whole.check() == 0
    ref = (mf.peaks_to_numpy(p), mf.triggers_to_numpy(t, n), int(n.item()))
    starts = shard.partition(m1, m2, [(N, spec.fs)], parts)
    outs = []
    for r in range(parts):
        b = shard.shard_bank(m1, m2, starts, r)
        pr, tr, nr = mf.filter_bank(b, [seg], 5.0, trig_cap=1 << 18)
        assert b.check() == 0
        outs.append(shard.local_results(b, pr, tr, nr))
    peaks, trig, n_all = shard.merge(outs)
    assert n_all == ref[2] and ref[2] > 0
    assert np.array_equal(peaks, ref[0])
    assert np.array_equal(trig, ref[1])
