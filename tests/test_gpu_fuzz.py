"""Seeded random machines of every shape against the oracle (needs a GPU).

Each case is one batch of a few hundred machines drawn from a fixed seed:
memory sizes 1..300 words (odd and even), programs of random length with
opcodes 0..9 (invalid ones halt), operands mixing small addresses, values
near n, negative and very large words, tapes shorter than or as long as the
capacity, step caps from 0 to a few hundred and none at all. Word sizes
cover the 4-byte layout (w <= 32) and the 8-byte one, and every schedule.
Every field of every machine, M included, must equal the oracle's.
"""
import numpy as np
import pytest

from paper_2604_12902_gb300 import workloads as W
from tests.helpers import U64, assert_same_state, oracle_state

pytestmark = pytest.mark.gpu

SCHEDS = {"auto": 0x00, "plain": 0x10, "staged": 0x20, "staged-step": 0x20020, "slab": 0x30, "vote": 0x130,
          "block": 0x20030}


@pytest.fixture(scope="module")
def rasp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12902_gb300 import rasp as R
    R.lib()
    return R


def random_batch(seed: int, w: int, num_vms: int = 400, ell: int = 5, s: int = 3) -> W.Workload:
    rng = np.random.default_rng(seed)
    ell, s = min(ell, (1 << w) - 1), min(s, (1 << w) - 1)        # l and s fit in w bits
    n = rng.integers(1, 301, size=num_vms)
    n[: num_vms // 8] = rng.integers(1, 9, size=num_vms // 8)          # some tiny memories
    progs, tapes = [], []
    for v in range(num_vms):
        m = int(rng.integers(0, n[v] // 2 + 1))                         # 2m <= n instructions' words
        # mostly valid opcodes, some invalid ones (0, 8, 9: the machine halts there)
        ops = np.where(rng.random(m) < 0.85, rng.integers(1, 8, size=m), rng.integers(0, 10, size=m))
        kind = rng.integers(0, 5, size=m)
        arg = np.where(kind == 0, rng.integers(0, n[v], size=m),
              np.where(kind == 1, rng.integers(-4, 4, size=m),
              np.where(kind == 2, n[v] + rng.integers(-2, 3, size=m),
              np.where(kind == 3, rng.integers(0, 2 * m + 1, size=m),
                       rng.integers(-(1 << 62), 1 << 62, size=m)))))
        p = np.empty(2 * m, np.int64)
        p[0::2] = ops
        p[1::2] = arg
        progs.append(p)
        tapes.append(rng.integers(-1000, 1000, size=int(rng.integers(0, ell + 1))).astype(np.int64))
    caps = rng.integers(0, 400, size=num_vms).astype(np.uint64)
    caps[rng.random(num_vms) < 0.3] = np.uint64(U64)
    po = np.zeros(num_vms + 1, np.uint64)
    po[1:] = np.cumsum([len(p) for p in progs])
    to = np.zeros(num_vms + 1, np.uint64)
    to[1:] = np.cumsum([len(t) for t in tapes])
    return W.Workload("fuzz", np.concatenate(progs) if po[-1] else np.zeros(0, np.int64), po,
                      n.astype(np.uint32), np.concatenate(tapes) if to[-1] else np.zeros(0, np.int64), to,
                      caps, ell, s, w)


BUDGET = 600      # some programs never halt: every run stops at this many steps


def check(R, wl, flags, semantics=0, what=""):
    st, _ = oracle_state(wl, budget=BUDGET, checked=semantics == 1, classic=bool(flags & 0x8000))
    with R.Batch(wl.mem_words, wl.ell, wl.s, word_bits=wl.w, flags=flags, semantics=semantics) as b:
        b.load_workload(wl)
        b.run(250)                    # resumed runs equal one run
        b.run(BUDGET)
        got = b.read_state()
    assert_same_state(got, st, wl.ell, wl.s, what=what)


@pytest.mark.parametrize("w", [2, 5, 13, 31, 32, 33, 50, 64])
@pytest.mark.parametrize("sched", list(SCHEDS))
def test_fuzz_word_machine(rasp, w, sched):
    check(rasp, random_batch(1000 + w, w), SCHEDS[sched], what="fuzz w %d %s" % (w, sched))


@pytest.mark.parametrize("w", [8, 32, 64])
@pytest.mark.parametrize("sched", ["plain", "slab"])
def test_fuzz_classic_opcode_set(rasp, w, sched):
    check(rasp, random_batch(2000 + w, w), SCHEDS[sched] | 0x8000, what="fuzz classic w %d %s" % (w, sched))


@pytest.mark.parametrize("sched", ["plain", "staged", "slab", "vote"])
def test_fuzz_checked_semantics(rasp, sched):
    check(rasp, random_batch(3000, 64), SCHEDS[sched], semantics=1, what="fuzz CHECKED %s" % sched)
