"""Multi-process sharding of a batch over ranks (CPU, gloo, world size 2).

Every rank generates its own disjoint shard of the template workload and runs
it through the oracle; nothing is exchanged but the final reduction. The
shards must partition the one-process workload exactly -- the same programs,
tapes and caps, VM by VM -- and the reduction must give the total VM-steps and
the slowest rank's time, as bench.py reports them."""
import os
import socket

import numpy as np
import pytest

from paper_2604_12902_gb300 import shards, workloads as W

PER_RANK = 384
WORLD = 2


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
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), steps=st.steps, status=st.status, i=st.i,
                 a=st.a, y=st.y, programs=wl.programs, tapes=wl.tapes, total_ms=ms, total_steps=steps)
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
    for p in parts:
        assert int(p["total_steps"]) == int(st.steps.sum())
        assert float(p["total_ms"]) == 10.0 + (WORLD - 1)


def test_shard_range_is_disjoint_and_contiguous():
    ranges = [shards.shard_range(r, 1000) for r in range(4)]
    assert ranges == [(0, 1000), (1000, 1000), (2000, 1000), (3000, 1000)]
    with pytest.raises(ValueError):
        shards.shard_range(-1, 10)
