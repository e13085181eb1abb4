"""Pins for the classic opcode set (Sec. 1.1: 3 = SUB, 5 = BPA) on the word
machine, in both oracle transcriptions. Hand evaluations of the two changed
cases (wraparound of SUB, the sign of a for BPA at w = 64 and w = 8), a
closed form for a SUB/BPA countdown, and brute-force agreement of the C
oracle with spec.py over every program of length <= 2 (and a sample of
length 3) on tiny memories."""
import numpy as np
import pytest

from oracle import oracle, spec
from tests.helpers import ADD, LOD, PRI, RD, STO, U64, asm, batch

SUB, BPA = 3, 5
APPLY, FIXED = 0, 1


def one(M, i=0, a=0, w=64, ell=2, s=2):
    return oracle.step_one(w, ell, s, i, a, [v & U64 for v in M], [0] * (ell + 1), [0] * (s + 1), classic=True)


def test_sub_wraps_modulo_2w():
    assert one([SUB, 3, 0, 10], a=15)[2] == 5
    assert one([SUB, 3, 0, 1], a=0)[2] == U64                     # 0 - 1 = 2^64 - 1
    assert one([SUB, 3, 0, 1], a=0, w=8)[2] == 255
    assert one([SUB, 3, 0, 200], a=100, w=8)[2] == (100 - 200) % 256


def test_bpa_jumps_only_on_positive_two_complement():
    prog = [BPA, 6, 0, 0, 0, 0, 0, 0]
    assert one(prog, a=1)[1] == 6
    assert one(prog, a=(1 << 63) - 1)[1] == 6                     # largest positive int64
    assert one(prog, a=0)[1] == 2
    assert one(prog, a=U64)[1] == 2                               # -1
    assert one(prog, a=1 << 63)[1] == 2                           # most negative int64
    assert one(prog, a=127, w=8)[1] == 6                          # w = 8: 127 > 0
    assert one(prog, a=128, w=8)[1] == 2                          # w = 8: 128 is -128
    assert one([BPA, 0, 0, 0], a=5)[0] == FIXED                   # jump to itself with a > 0
    assert one([BPA, 0, 0, 0], a=U64)[0] == APPLY                 # a < 0: falls through


def test_other_opcodes_are_the_word_machine():
    for M, a in (([LOD, 42, 0, 0], 7), ([ADD, 3, 0, 10], 5), ([STO, 3, 0, 0], 9), ([PRI, 3, 0, 4], 0)):
        assert one(M, a=a) == oracle.step_one(64, 2, 2, 0, a, [v & U64 for v in M], [0] * 3, [0] * 3)
    got = oracle.step_one(64, 2, 2, 0, 0, [RD, 3, 0, 0], [0, 11, 22], [0, 0, 0], classic=True)
    assert got[3] == [RD, 3, 0, 11]


def countdown(T):
    # one <- 1; a <- T; loop: a <- a - one; if a > 0 goto loop; print one; halt
    return asm((LOD, 1), (STO, 30), (LOD, T), (SUB, 30), (BPA, 6), (PRI, 30), (0, 0))


@pytest.mark.parametrize("T", [1, 2, 3, 10, 100, 0, -1, -100])
def test_countdown_closed_form(T):
    # hand count: LOD, STO, LOD (3); T pairs SUB/BPA while T >= 1, else one pair; PRI (1)
    want = 3 + 2 * max(T, 1) + 1
    p, po, nn, t, to, caps = batch([countdown(T)], [[]], 40)
    st, _ = oracle.run_packed(p, po, nn, t, to, 0, 2, classic=True)
    assert int(st.status[0]) == 1 and int(st.steps[0]) == want
    assert int(st.y[1]) == 1 and int(st.a[0]) == (min(T, 1) - 1) % (1 << 64)
    c, steps, status = spec.run(spec.initial(countdown(T), [], 40, 0, 2, 64), 0, 2, 64, 10 ** 6, classic=True)
    assert (steps, status) == (want, 1)


def test_countdown_differs_from_the_word_machine():
    # the same words on the word machine: opcode 3 multiplies, opcode 5 tests a != 0
    p, po, nn, t, to, caps = batch([countdown(5)], [[]], 40, 1000)
    word, _ = oracle.run_packed(p, po, nn, t, to, 0, 2, caps=caps)
    cls, _ = oracle.run_packed(p, po, nn, t, to, 0, 2, caps=caps, classic=True)
    assert int(word.status[0]) == 2 and int(word.steps[0]) == 1000      # 5 x 1 stays 5: loops
    assert int(cls.status[0]) == 1 and int(cls.steps[0]) == 14


OPS = list(range(9))
ARGS = [0, 1, 2, 5, 1 << 63, U64]


def _compare(programs, n, tape, w, cap=64, ell=2, s=2):
    p, po, nn, t, to, caps = batch(programs, [tape] * len(programs), n, cap)
    st, _ = oracle.run_packed(p, po, nn, t, to, ell, s, caps=caps, w=w, classic=True)
    for v, prog in enumerate(programs):
        c, steps, status = spec.run(spec.initial(prog, tape, n, ell, s, w), ell, s, w, cap, classic=True)
        assert (int(st.steps[v]), int(st.status[v])) == (steps, status), (prog, w)
        assert int(st.i[v]) == c[0] and int(st.a[v]) == c[1]
        assert [int(q) for q in st.memory(v)] == list(c[2])
        assert [int(q) for q in st.y[v * (s + 1):(v + 1) * (s + 1)]] == list(c[4])


@pytest.mark.parametrize("n", [6, 8])
@pytest.mark.parametrize("tape", [[], [3, -2]])
@pytest.mark.parametrize("w", [64, 8, 2])
def test_exhaustive_length_le_2_matches_spec(n, tape, w):
    instrs = [(o, a) for o in OPS for a in ARGS]
    progs = [[]] + [asm(x) for x in instrs] + [asm(x, y) for x in instrs for y in instrs]
    _compare(progs, n, tape, w)


def test_length_3_sample_matches_spec():
    instrs = [(o, a) for o in OPS for a in ARGS]
    rng = np.random.default_rng(4)
    picks = rng.integers(0, len(instrs), size=(20000, 3))
    progs = [asm(*(instrs[k] for k in row)) for row in picks]
    _compare(progs, 6, [3, -2], 64)
    _compare(progs[:6000], 8, [], 8)
