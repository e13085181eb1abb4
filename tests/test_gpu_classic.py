"""The classic opcode set (Sec. 1.1: 3 = SUB, 5 = BPA with a > 0) on the GPU,
bit-exact against the oracle run with the same opcode set. Needs a GPU."""
import os

import numpy as np
import pytest

from paper_2604_12902_gb300 import workloads as W
from tests.helpers import ADD, LOD, PRI, RD, STO, U64, asm, assert_same_state, batch, oracle_state

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1
SUB, BPA = 3, 5
SCHEDS = {"plain": 0x10, "persist_gl": 0x30, "auto": 0x00}


@pytest.fixture(scope="module")
def rasp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12902_gb300 import rasp as R
    R.lib()
    return R


def run_gpu(R, wl, flags, budget=U64, semantics=0, split=None):
    with R.Batch(wl.mem_words, wl.ell, wl.s, word_bits=wl.w, semantics=semantics,
                 flags=flags | R.ISA_CLASSIC) as b:
        b.load_workload(wl)
        for t in split or []:
            b.run(t)
        b.run(budget)
        return b.read_state(), b.stats()


def wl_from(programs, tapes, n, caps, ell, s, w=64):
    p, po, nn, t, to, cc = batch(programs, tapes, n, caps)
    return W.Workload("classic", p, po, nn.astype(np.uint32), t, to,
                      cc if cc is not None else np.full(len(programs), U64, np.uint64), ell, s, w)


@pytest.mark.parametrize("sched", list(SCHEDS))
@pytest.mark.parametrize("w", [64, 8])
def test_random_programs(rasp, sched, w):
    wl = W.random_programs(num_vms=20000, seed=31)
    wl.w = w
    st, _ = oracle_state(wl, threads=THREADS, classic=True)
    got, stats = run_gpu(rasp, wl, SCHEDS[sched])
    assert_same_state(got, st, wl.ell, wl.s, what="classic random %s w=%d" % (sched, w))
    word, _ = oracle_state(wl, threads=THREADS)
    assert not np.array_equal(word.steps, st.steps)          # the opcode set matters


@pytest.mark.parametrize("n,tape,w", [(6, [3, -2], 64), (8, [], 8), (6, [], 2)])
def test_exhaustive_tiny_programs(rasp, n, tape, w):
    ops, args = list(range(9)), [0, 1, 2, 5, 1 << 63, U64]
    instrs = [(o, a) for o in ops for a in args]
    progs = [asm(x, y) for x in instrs for y in instrs]
    rng = np.random.default_rng(9)
    progs += [asm(*(instrs[k] for k in row)) for row in rng.integers(0, len(instrs), size=(40000, 3))]
    wl = wl_from(progs, [tape] * len(progs), n, 64, 2, 2, w=w)
    st, _ = oracle_state(wl, threads=THREADS, classic=True)
    for sched in ("plain", "persist_gl"):
        got, _ = run_gpu(rasp, wl, SCHEDS[sched])
        assert_same_state(got, st, 2, 2, what="classic exhaustive %s n=%d w=%d" % (sched, n, w))


def test_countdowns_across_budget_rounds(rasp):
    """SUB/BPA countdowns of up to ~200,000 steps (closed form 4 + 2 max(T, 1)),
    some capped, in one run and split at budgets inside the rounds."""
    rng = np.random.default_rng(5)
    Ts = rng.integers(-50, 100_000, size=3000)
    progs = [asm((LOD, 1), (STO, 30), (LOD, int(T)), (SUB, 30), (BPA, 6), (PRI, 30), (0, 0)) for T in Ts]
    caps = rng.integers(100, 250_000, size=len(progs)).astype(np.uint64)
    caps[::5] = U64
    wl = wl_from(progs, [[]] * len(progs), 40, caps, 0, 2)
    st, _ = oracle_state(wl, threads=THREADS, classic=True)
    halted = st.status == 1
    assert np.array_equal(st.steps[halted], (4 + 2 * np.maximum(Ts, 1))[halted].astype(np.uint64))
    for split in (None, [5_000, 40_000, 100_001]):
        got, _ = run_gpu(rasp, wl, SCHEDS["persist_gl"] | rasp.BUDGET_ROUNDS, split=split)
        assert_same_state(got, st, 0, 2, what="classic countdown split=%s" % split)


def test_checked_subtraction_overflow(rasp):
    big, small = (1 << 63) - 5, -(1 << 63) + 5
    progs = [asm((RD, 20), (RD, 21), (LOD, 0), (ADD, 20), (SUB, 21), (PRI, 20), (0, 0)),
             asm((RD, 20), (LOD, 0), (SUB, 20), (SUB, 20), (0, 0)),
             asm((RD, 20), (RD, 21), (LOD, 0), (ADD, 20), (SUB, 21), (0, 0))]
    tapes = [[small, 10], [small, 0], [big, -10]]
    wl = wl_from(progs, tapes, 24, None, 2, 2)
    st, _ = oracle_state(wl, checked=True, classic=True)
    assert list(st.status) == [3, 3, 3]
    for sched in ("plain", "persist_gl"):
        got, _ = run_gpu(rasp, wl, SCHEDS[sched], semantics=rasp.CHECKED)
        assert_same_state(got, st, 2, 2, what="classic checked %s" % sched)


def test_autotune_and_rejected_configurations(rasp):
    wl = W.random_programs(num_vms=5000, seed=8)
    st, _ = oracle_state(wl, threads=THREADS, classic=True)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, flags=rasp.ISA_CLASSIC) as b:
        b.load_workload(wl)
        rep = b.autotune(reps=1)
        assert all(t["schedule"].startswith(("persist_gl", "plain")) for t in rep["trials"])
        b.run()
        assert_same_state(b.read_state(), st, wl.ell, wl.s, what="classic autotuned")
    for flags in (0x20 | rasp.ISA_CLASSIC, 0x40 | rasp.ISA_CLASSIC, 0x100 | rasp.ISA_CLASSIC):
        with pytest.raises(rasp.RaspError) as e:
            rasp.Batch(wl.mem_words, wl.ell, wl.s, flags=flags)
        assert e.value.code == rasp.RASP_EINVAL


def test_templates_full_size_classic(rasp):
    """The classic-opcode benchmark workload (1,048,576 template programs,
    n = 256, cap 4096) in its launch configuration: every VM against the
    oracle run with the classic opcode set."""
    wl = W.template_programs(num_vms=1 << 20, seed=2)
    st, _ = oracle_state(wl, threads=THREADS, classic=True)
    got, stats = run_gpu(rasp, wl, 0)
    assert_same_state(got, st, wl.ell, wl.s, what="classic templates full")
    assert stats["halted"] == int((st.status == 1).sum())
    assert stats["vm_steps"] == int(st.steps.sum())
