"""Multi-process sharding of a batch over ranks (CPU, gloo, world size 2).

Every rank generates its own disjoint shard of the template workload and runs
it through the oracle; nothing is exchanged but the final reduction. The
shards must partition the one-process workload exactly -- the same programs,
tapes and caps, VM by VM -- and the reductions must give the total VM-steps,
the slowest rank's time (as bench.py reports them) and the whole batch's
tau_h histogram."""
import os
import socket

import numpy as np
import pytest

from paper_2604_12902_gb300 import shards, workloads as W

PER_RANK = 384
WORLD = 2
HIST_BINS = 4097       # template VMs take at most 4096 steps


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    from oracle import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, count = shards.shard_range(rank, PER_RANK)
        wl = W.template_programs(num_vms=count, seed=2, first_vm=first)
        st, _ = oracle.run_packed(wl.programs, wl.prog_off, wl.mem_words, wl.tapes, wl.tape_off,
                                  wl.ell, wl.s, caps=wl.caps)
        fake_ms = 10.0 + rank                      # the slowest rank's time must win
        ms, steps = shards.combine(dist, fake_ms, int(st.steps.sum()))
        hist = shards.combine_counts(dist, np.bincount(st.steps.astype(np.int64), minlength=HIST_BINS)[:HIST_BINS])
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), steps=st.steps, status=st.status, i=st.i,
                 a=st.a, y=st.y, programs=wl.programs, tapes=wl.tapes, total_ms=ms, total_steps=steps,
                 hist=hist)
    finally:
        dist.destroy_process_group()


def test_shards_partition_the_workload_and_reduce(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(WORLD, _free_port(), str(tmp_path)), nprocs=WORLD,
                       start_method="spawn", join=True)
    from oracle import oracle
    whole = W.template_programs(num_vms=WORLD * PER_RANK, seed=2)
    st, _ = oracle.run_packed(whole.programs, whole.prog_off, whole.mem_words, whole.tapes, whole.tape_off,
                              whole.ell, whole.s, caps=whole.caps)
    parts = [np.load(os.path.join(tmp_path, "rank%d.npz" % r)) for r in range(WORLD)]
    np.testing.assert_array_equal(np.concatenate([p["programs"] for p in parts]), whole.programs)
    np.testing.assert_array_equal(np.concatenate([p["tapes"] for p in parts]), whole.tapes)
    for key in ("steps", "status", "i", "a", "y"):
        np.testing.assert_array_equal(np.concatenate([p[key] for p in parts]), getattr(st, key), err_msg=key)
    want_hist = np.bincount(st.steps.astype(np.int64), minlength=HIST_BINS)[:HIST_BINS]
    for p in parts:
        assert int(p["total_steps"]) == int(st.steps.sum())
        assert float(p["total_ms"]) == 10.0 + (WORLD - 1)
        np.testing.assert_array_equal(p["hist"], want_hist)


def test_shard_range_is_disjoint_and_contiguous():
    ranges = [shards.shard_range(r, 1000) for r in range(4)]
    assert ranges == [(0, 1000), (1000, 1000), (2000, 1000), (3000, 1000)]
    with pytest.raises(ValueError):
        shards.shard_range(-1, 10)


def _best_bottleneck(c, k):
    """Smallest possible largest range cost over all splits of c into at most
    k contiguous ranges (brute force by dynamic programming)."""
    import functools
    pre = np.concatenate([[0], np.cumsum(c)])

    @functools.lru_cache(maxsize=None)
    def f(i, k):
        if i == len(c):
            return 0
        if k == 0:
            return float("inf")
        return min(max(int(pre[j] - pre[i]), f(j, k - 1)) for j in range(i + 1, len(c) + 1))
    return f(0, k)


def test_balanced_ranges_are_optimal_contiguous_splits():
    rng = np.random.default_rng(5)
    for _ in range(300):
        V = int(rng.integers(1, 13))
        k = int(rng.integers(1, 5))
        c = rng.integers(0, 50, size=V)
        r = shards.balanced_ranges(c, k)
        assert len(r) == k
        assert r[0][0] == 0 and all(a[0] + a[1] == b[0] for a, b in zip(r, r[1:]))
        assert r[-1][0] + r[-1][1] == V
        worst = max(int(c[f:f + n].sum()) for f, n in r)
        assert worst == _best_bottleneck(tuple(int(x) for x in c), k)


def test_balanced_ranges_on_the_uneven_batch():
    """Caps of the uneven batch vary over three orders of magnitude: balanced
    ranges differ from equal counts and cut the largest shard's cap sum."""
    wl = W.uneven_programs(num_vms=4096, seed=3)
    cost = shards.estimated_cost(wl)
    r = shards.balanced_ranges(cost, 4)
    worst = max(int(cost[f:f + n].sum()) for f, n in r)
    equal = max(int(cost[k * 1024:(k + 1) * 1024].sum()) for k in range(4))
    assert worst <= equal and worst - int(cost.sum()) / 4 <= int(cost.max())
    sub = W.uneven_programs(num_vms=r[2][1], seed=3, first_vm=r[2][0])
    assert np.array_equal(sub.caps, wl.caps[r[2][0]:r[2][0] + r[2][1]])
