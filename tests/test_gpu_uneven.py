"""Uneven batches: mixed program lengths, memory sizes (odd n, non powers of
two, 16..4096 words) and step caps, about 30% non-halting; bucketing, merged
launches, longest-cap-first order and CUDA-graph replay (needs a GPU)."""
import os

import numpy as np
import pytest

from paper_2604_12902_gb300 import workloads as W
from tests.helpers import U64, assert_same_state, oracle_state

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def rasp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12902_gb300 import rasp as R
    R.lib()
    return R


@pytest.fixture(scope="module")
def uneven64k():
    wl = W.uneven_programs(num_vms=1 << 16, seed=3)
    st, _ = oracle_state(wl, threads=THREADS)
    return wl, st


@pytest.mark.parametrize("flags", [0x00, 0x10, 0x20, 0x30, 0x4000, 0x4030, 0x130])
def test_uneven_batch_every_vm(rasp, uneven64k, flags):
    wl, st = uneven64k
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, flags=flags) as b:
        b.load_workload(wl)
        b.run()
        got = b.read_state()
        if flags & 0x4000:                       # replay the captured graph on a fresh c_0
            b.reset()
            b.run()
            again = b.read_state()
            for k in got:
                assert np.array_equal(got[k], again[k]), k
    assert_same_state(got, st, wl.ell, wl.s, what="uneven flags=%#x" % flags)
    counts = np.bincount(st.status, minlength=5)
    assert 0.2 < counts[2] / wl.num_vms < 0.45           # about 30% time out


def test_graph_replay_with_budgets(rasp, uneven64k):
    wl, full = uneven64k
    part, _ = oracle_state(wl, budget=300, threads=THREADS)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, flags=0x4000) as b:
        b.load_workload(wl)
        b.run(300)
        got = b.read_state()
        assert_same_state(got, part, wl.ell, wl.s, what="graph budget 300")
        b.run()
        got = b.read_state()
        assert_same_state(got, full, wl.ell, wl.s, what="graph resumed")
        assert b.describe()["cuda_graph"] is True


def test_auto_schedule_merges_buckets_into_one_launch_group(rasp, uneven64k):
    """All memory buckets run in one persistent launch group: 65,536 VMs fit
    the resident lanes, so one launch; with RASP_BUDGET_ROUNDS the group runs
    in budget rounds (4096, x8, ... below the largest cap, then the run's
    budget), each round after the first preceded by a compaction launch."""
    wl, full = uneven64k
    with rasp.Batch(wl.mem_words, wl.ell, wl.s) as b:
        d = b.describe()
        assert len(d["buckets"]) >= 5
        assert len(d["launches"]) == 1 and d["launches"][0]["vms"] == wl.num_vms
        b.load_workload(wl)
        b.run()
        assert b.stats()["launches"] == 1
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, flags=rasp.BUDGET_ROUNDS) as b:
        b.load_workload(wl)
        b.run()
        rounds, r = 1, 4096
        while r < int(wl.caps.max()) and rounds <= 6:
            rounds, r = rounds + 1, r * 8
        assert b.stats()["launches"] == 1 + 2 * (rounds - 1)
        got = b.read_state()
    assert_same_state(got, full, wl.ell, wl.s, what="uneven with budget rounds")


def test_uneven_full_size_sampled(rasp):
    """4,194,304 programs (about 28 GiB of M): every VM checked for the
    invariants, 3,000 sampled VMs compared with the oracle field by field."""
    wl = W.uneven_programs(num_vms=1 << 22, seed=3, workers=THREADS)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, flags=0x4000) as b:
        b.load_workload(wl)
        b.run()
        got = b.read_state(mem=False)
        stats = b.stats()
        rng = np.random.default_rng(33)
        ids = np.sort(rng.choice(wl.num_vms, size=3000, replace=False))
        mems = [b.read_state(first=int(v), count=1)["mem"] for v in ids]
    assert np.all(got["steps"] <= wl.caps)
    assert set(np.unique(got["status"])) <= {1, 2}
    to = got["status"] == 2
    assert np.all(got["steps"][to] == wl.caps[to])
    assert 0.2 < to.mean() < 0.45
    assert stats["vm_steps"] == int(got["steps"].sum())
    sub = wl.subset(ids)
    st, _ = oracle_state(sub, threads=THREADS)
    sel = {k: got[k][ids] for k in ("i", "a", "steps", "status", "uhead", "ylen", "y")}
    sel["mem"] = np.concatenate(mems)
    assert_same_state(sel, st, wl.ell, wl.s, what="uneven full-size sample")


def test_autotune_leaves_state_and_keeps_parity(rasp, uneven64k):
    wl, st = uneven64k
    with rasp.Batch(wl.mem_words, wl.ell, wl.s) as b:
        b.load_workload(wl)
        b.run(50)
        before = b.read_state()
        rep = b.autotune(reps=1)
        after = b.read_state()
        for k in before:
            assert np.array_equal(before[k], after[k]), k
        assert len(rep["trials"]) == 9          # no shared candidate: programs not shared
        assert rep["chosen"] in [t["schedule"] for t in rep["trials"]]
        best = min(rep["trials"], key=lambda t: t["ms"])
        assert rep["chosen"] == best["schedule"]
        # the per-bucket pass: one entry per non-empty bucket, each choice one
        # of its trials or the global choice; pinned buckets show in the plan
        plan = b.describe()
        assert len(rep["buckets"]) == len(plan["buckets"]) > 1
        for entry in rep["buckets"]:
            names = [t["schedule"] for t in entry["trials"]]
            assert entry["chosen"] in names + [rep["chosen"]]
            assert rep["chosen"] not in names
        pinned = sum(e["chosen"] != rep["chosen"] for e in rep["buckets"])
        assert sum(k["pinned"] for k in plan["buckets"]) == pinned
        assert rep["per_bucket_ms"] <= best["ms"]
        b.run()
        got = b.read_state()
    assert_same_state(got, st, wl.ell, wl.s, what="after autotune (%s)" % rep["chosen"])


PLAIN, PERSIST, PERSIST_GL, AUTO = 0x10, 0x20, 0x30, 0x00


@pytest.mark.parametrize("flags", [0x00, 0x4000], ids=["eager", "cuda-graph"])
def test_pinned_bucket_schedules_every_vm(rasp, uneven64k, flags):
    """Every memory-size bucket on a schedule of its own (plain, SMEM-staged,
    HBM-slab with 3 or 5 resident CTAs per SM and 2-warp CTAs, batch-wide):
    separate launches per bucket, every VM equal to the oracle's, with
    budget rounds, resumed runs and graph replay."""
    wl, st = uneven64k
    choices = [(PLAIN, 0, 0, 0), (PERSIST, 32, 1, 0), (PERSIST_GL, 128, 4, 3), (PERSIST_GL, 64, 2, 5), (AUTO, 0, 0, 0)]
    part, _ = oracle_state(wl, budget=3000, threads=THREADS)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, flags=flags | rasp.BUDGET_ROUNDS) as b:
        b.load_workload(wl)
        buckets = b.describe()["buckets"]
        assert len(buckets) > 3
        for j, k in enumerate(buckets):
            b.plan_bucket(k["index"], *choices[j % len(choices)])
        plan = b.describe()
        assert [k["pinned"] for k in plan["buckets"]] == [choices[j % len(choices)][0] != AUTO
                                                         for j in range(len(buckets))]
        assert len(plan["launches"]) > 3
        b.run(3000)
        assert_same_state(b.read_state(), part, wl.ell, wl.s, what="pinned buckets, budget 3000")
        b.run()
        assert_same_state(b.read_state(), st, wl.ell, wl.s, what="pinned buckets, resumed")
        b.reset()
        b.run(3000)
        b.run()
        assert_same_state(b.read_state(), st, wl.ell, wl.s, what="pinned buckets, after reset")
        with pytest.raises(rasp.RaspError):
            b.plan_bucket(99, PLAIN)
        with pytest.raises(rasp.RaspError):
            b.plan_bucket(0, 0x40)
