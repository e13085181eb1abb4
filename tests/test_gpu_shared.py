"""Shared-program schedule: one program in shared memory per CTA, many VMs
(inputs) per program, copy-on-write when a VM writes into its program words
(needs a GPU)."""
import os

import numpy as np
import pytest

from paper_2604_12902_gb300 import workloads as W
from tests.helpers import assert_same_state, oracle_state

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1
SHARED = 0x40


@pytest.fixture(scope="module")
def rasp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12902_gb300 import rasp as R
    R.lib()
    return R


def run(R, wl, flags, budgets=(None,)):
    with R.Batch(wl.mem_words, wl.ell, wl.s, word_bits=wl.w, flags=flags) as b:
        b.load_workload(wl)
        for t in budgets:
            b.run() if t is None else b.run(t)
        return b.read_state(), b.stats()


def self_modifying_shared(P=300, R=40, seed=8):
    """Random 32-instruction programs filling a 64-word memory (STO and RD
    land on code often), shared by R VMs each."""
    base = W.random_programs(num_vms=P, seed=seed)
    V = P * R
    ids = np.arange(V, dtype=np.uint64)
    tape = W.uniform_int(W.draws(seed, 9, ids, 4), -100, 100).reshape(-1)
    return W.Workload("selfmod-shared", base.programs, base.prog_off, np.full(V, 64, np.uint32), tape,
                      np.arange(V + 1, dtype=np.uint64) * 4, np.full(V, 256, np.uint64), 4, 8,
                      prog_of_vm=np.repeat(np.arange(P, dtype=np.uint32), R))


def test_shared_templates_every_vm(rasp):
    wl = W.shared_programs(num_programs=512, vms_per_program=64)
    st, _ = oracle_state(wl, threads=THREADS)
    got, stats = run(rasp, wl, SHARED)
    assert_same_state(got, st, wl.ell, wl.s, what="shared templates")
    assert stats["halted"] == wl.num_vms


def test_shared_self_modifying_code(rasp):
    wl = self_modifying_shared()
    st, _ = oracle_state(wl, threads=THREADS)
    got, _ = run(rasp, wl, SHARED)
    assert_same_state(got, st, wl.ell, wl.s, what="shared self-modifying")
    part, _ = oracle_state(wl, budget=37, threads=THREADS)
    got, _ = run(rasp, wl, SHARED, budgets=(37,))
    assert_same_state(got, part, wl.ell, wl.s, what="shared self-modifying, budget 37")
    got, _ = run(rasp, wl, SHARED, budgets=(5, 37, 90, None))
    assert_same_state(got, st, wl.ell, wl.s, what="shared self-modifying, resumed")


def test_shared_after_other_schedule_and_autotune(rasp):
    wl = self_modifying_shared(P=100, R=20, seed=9)
    st, _ = oracle_state(wl, threads=THREADS)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, flags=0x30) as b:       # persistent, then shared
        b.load_workload(wl)
        b.run(20)
        before = b.read_state()
        rep = b.autotune(reps=1)
        assert "shared" in [t["schedule"] for t in rep["trials"]]
        after = b.read_state()
        for k in before:
            assert np.array_equal(before[k], after[k]), k
        b.run()
        got = b.read_state()
    assert_same_state(got, st, wl.ell, wl.s, what="after autotune (%s)" % rep["chosen"])


def test_shared_masked_word_size(rasp):
    wl = W.shared_programs(num_programs=64, vms_per_program=32, seed=6)
    wl.w = 16
    st, _ = oracle_state(wl)
    got, _ = run(rasp, wl, SHARED)
    assert_same_state(got, st, wl.ell, wl.s, what="shared w=16")


def test_shared_full_size_sampled(rasp):
    """16,384 programs x 256 tapes = 4,194,304 VMs; every VM halts; 2,000
    sampled VMs compared with the oracle."""
    wl = W.shared_programs()
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, flags=SHARED) as b:
        b.load_workload(wl)
        b.run()
        got = b.read_state(mem=False)
        stats = b.stats()
        ids = np.sort(np.random.default_rng(44).choice(wl.num_vms, size=2000, replace=False))
        mems = [b.read_state(first=int(v), count=1)["mem"] for v in ids]
    assert stats["halted"] == wl.num_vms
    sub = wl.subset(ids)
    st, _ = oracle_state(sub, threads=THREADS)
    sel = {k: got[k][ids] for k in ("i", "a", "steps", "status", "uhead", "ylen", "y")}
    sel["mem"] = np.concatenate(mems)
    assert_same_state(sel, st, wl.ell, wl.s, what="shared full-size sample")


STEP_BLOCK, COLLECT_STATS = 0x20000, 0x1000


@pytest.mark.parametrize("extra", [0, STEP_BLOCK, COLLECT_STATS], ids=["epoch-loop", "per-step", "counters"])
def test_shared_forms_every_vm(rasp, extra):
    """The three shared-program kernels (the epoch loop, and the one-step
    form with and without counters) against the oracle, on templates and on
    self-modifying code that writes into the shared program words."""
    for wl in (W.shared_programs(num_programs=256, vms_per_program=32, seed=12), self_modifying_shared(P=150, R=24)):
        st, _ = oracle_state(wl, threads=THREADS)
        got, _ = run(rasp, wl, SHARED | extra)
        assert_same_state(got, st, wl.ell, wl.s, what="shared %s flags %#x" % (wl.name, extra))


def test_shared_checked_semantics(rasp):
    """CHECKED semantics on the shared-program schedule (one-step form)."""
    wl = self_modifying_shared(P=120, R=16, seed=13)
    st, _ = oracle_state(wl, checked=True, threads=THREADS)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, semantics=rasp.CHECKED, flags=SHARED) as b:
        b.load_workload(wl)
        b.run()
        got = b.read_state()
    assert_same_state(got, st, wl.ell, wl.s, what="shared CHECKED")


def test_shared_lazy_pack_read_back_midway(rasp):
    """c_0 of the shared-program schedule writes only data words; reading M
    back fills in the program words first. Reading midway, running on,
    resetting and running again all match the oracle."""
    wl = self_modifying_shared(P=120, R=16, seed=11)
    part, _ = oracle_state(wl, budget=30, threads=THREADS)
    st, _ = oracle_state(wl, threads=THREADS)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, flags=SHARED) as b:
        b.load_workload(wl)
        b.run(30)
        assert_same_state(b.read_state(), part, wl.ell, wl.s, what="lazy pack, read at 30 steps")
        b.run()
        assert_same_state(b.read_state(), st, wl.ell, wl.s, what="lazy pack, run on after the read")
        b.reset()
        b.run(30)
        assert_same_state(b.read_state(mem=False), part, wl.ell, wl.s, what="lazy pack again, no M read")
        b.run()
        assert_same_state(b.read_state(), st, wl.ell, wl.s, what="lazy pack again, run to the end")


def test_shared_lazy_pack_checkpoint_restore(rasp):
    """A checkpoint taken on one lazily packed batch, restored into another
    lazily packed batch midway through its own run, then run on."""
    wl = self_modifying_shared(P=100, R=12, seed=14)
    st, _ = oracle_state(wl, threads=THREADS)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, flags=SHARED) as b1, \
            rasp.Batch(wl.mem_words, wl.ell, wl.s, flags=SHARED) as b2:
        b1.load_workload(wl)
        b1.run(25)
        ck = b1.read_state()
        b2.load_workload(wl)
        b2.run(7)
        half = wl.num_vms // 2
        b2.load_state({k: v[:half] for k, v in ck.items() if k != "mem"} |
                      {"mem": ck["mem"][:int(wl.mem_words[:half].astype(np.uint64).sum())]})
        b2.run()
        got = b2.read_state()
    assert_same_state(got, st, wl.ell, wl.s, what="restored halves then run on")


def test_shared_lazy_pack_through_autotune(rasp):
    """Autotuning a lazily packed batch: its non-shared trials fill in the
    program words, the state is put back as it was (lazy), and the batch
    then runs to the oracle's result on whichever schedule was chosen."""
    wl = self_modifying_shared(P=100, R=20, seed=15)
    st, _ = oracle_state(wl, threads=THREADS)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, flags=SHARED) as b:
        b.load_workload(wl)
        b.run(20)
        before = b.read_state(mem=False)
        rep = b.autotune(reps=1)
        after = b.read_state(mem=False)
        for k in before:
            assert np.array_equal(before[k], after[k]), k
        b.run()
        got = b.read_state()
    assert_same_state(got, st, wl.ell, wl.s, what="lazy pack through autotune (%s)" % rep["chosen"])
