"""Pins for the CPU oracle against what the paper and arithmetic fix.

Each test states its source: a hand evaluation of one case of the Sec. 2.1
transition, a closed form derived by hand for a small program, the halting
numbers printed in App. B, or brute-force agreement with the independent
pure-Python transcription in ``oracle/spec.py``.
"""
import numpy as np
import pytest

from oracle import oracle, spec
from paper_2604_12902_gb300 import dsl
from tests.helpers import (ADD, BNZ, HLT, LOD, MUL, PRI, RD, STO, U64, asm, batch,
                           busy_beavers)

APPLY, FIXED, FAULT_ADDR_K, FAULT_OVF_K = 0, 1, 2, 3


def one(M, i=0, a=0, u=(0, 0, 0), y=(0, 0, 0), ell=2, s=2, w=64, checked=False):
    return oracle.step_one(w, ell, s, i, a, [v & U64 for v in M], list(u), list(y), checked=checked)


# ------------------------------------------------------------ single cases
def test_lod_is_immediate():
    k, i, a, M, u, y = one([LOD, 42, 0, 0], a=7)
    assert (k, i, a, M) == (APPLY, 2, 42, [1, 42, 0, 0])
    k, i, a, *_ = one([LOD, -5, 0, 0])
    assert a == U64 - 4


def test_add_mul_and_wraparound():
    assert one([ADD, 3, 0, 10], a=5)[2] == 15
    assert one([ADD, 3, 0, 1], a=U64)[2] == 0                       # (2^64-1) + 1 = 0
    assert one([MUL, 3, 0, 7], a=6)[2] == 42
    assert one([MUL, 3, 0, 1 << 32], a=1 << 32)[2] == 0             # 2^64 = 0
    assert one([MUL, 3, 0, 5], a=U64 - 2)[2] == (-15) & U64           # -3 * 5


def test_sto_and_circular_operand():
    k, i, a, M, *_ = one([STO, 3, 0, 0], a=9)
    assert M == [4, 3, 0, 9] and i == 2 and a == 9
    k, i, a, M, *_ = one([STO, 7, 0, 0], a=9)                        # 7 mod 4 = 3
    assert M == [4, 7, 0, 9]


def test_operand_mod_is_unsigned():
    # j = -1 is the word 2^64-1; (2^64-1) mod 250 = 115 (floored signed mod would give 249)
    M = [0] * 250
    M[0], M[1], M[115], M[249] = ADD, -1, 1000, 5
    assert one(M, a=1)[2] == 1001


def test_fetch_wraps_at_word_boundary():
    # i = 2^64-1: o = M[i mod 250] = M[115], j = M[(i (+) 1) mod 250] = M[0]
    M = [0] * 250
    M[115], M[0], M[116] = LOD, 77, 55
    k, i, a, *_ = one(M, i=U64)
    assert (k, a, i) == (APPLY, 77, 1)                                # i (+) 2 = 1


def test_fetch_circular_at_last_word():
    M = [55, 0, 0, 0, LOD]                                            # i = 4: o = M[4], j = M[0]
    k, i, a, *_ = one(M, i=4)
    assert (k, i, a) == (APPLY, 6, 55)


def test_bnz():
    assert one([BNZ, 6, 0, 0, 0, 0, 0, 0], a=1)[1] == 6
    assert one([BNZ, 6, 0, 0, 0, 0, 0, 0], a=0)[1] == 2
    assert one([BNZ, 0, 0, 0], a=1)[0] == FIXED                       # self-jump: c -> c
    # j = 4 is congruent to i = 0 mod 4 but differs from i: one more step, then a fixed point
    k, i, *_ = one([BNZ, 4, 0, 0], a=1)
    assert (k, i) == (APPLY, 4)
    assert one([BNZ, 4, 0, 0], i=4, a=1)[0] == FIXED


def test_rd_reads_then_halts_on_exhaustion():
    k, i, a, M, u, y = one([RD, 3, 0, 0], u=(0, 11, 22))
    assert (k, i, M, u) == (APPLY, 2, [6, 3, 0, 11], [1, 11, 22])
    k, i, a, M, u, y = one([RD, 3, 0, 0], u=(1, 11, 22))
    assert (M, u) == ([6, 3, 0, 22], [2, 11, 22])
    assert one([RD, 3, 0, 0], u=(2, 11, 22))[0] == FIXED             # u_0 = l: "otherwise"


def test_pri_appends_until_full_and_advances_when_full():
    k, i, a, M, u, y = one([PRI, 3, 0, 99])
    assert (k, i, y) == (APPLY, 2, [1, 99, 0])
    k, i, a, M, u, y = one([PRI, 3, 0, 99], y=(2, 5, 6))
    assert (k, i, y) == (APPLY, 2, [2, 5, 6])                          # y :: z = y, i still moves


@pytest.mark.parametrize("op", [0, 8, 9, 1 << 63, U64])
def test_invalid_opcodes_are_fixed_points(op):
    assert one([op, 1, 0, 0], a=3)[0] == FIXED


def test_word_size_masking():
    k, i, a, *_ = one([ADD, 3, 0, 100], a=200, w=8)
    assert a == 44                                                    # 300 mod 256
    M = [0] * 256
    M[254], M[255] = LOD, 7
    assert one(M, i=254, w=8)[1] == 0                                 # 254 (+) 2 = 0 mod 2^8


# ------------------------------------------------------------ CHECKED mode
# No counterpart in the paper: these pin the written rule (fetch range, then
# fixed point, then operand range, then signed overflow).
def test_checked_faults():
    big = (1 << 63) - 1
    assert one([ADD, 3, 0, 1], a=big, checked=True)[0] == FAULT_OVF_K
    assert one([ADD, 3, 0, 1], a=big - 1, checked=True)[0] == APPLY
    assert one([ADD, 3, 0, U64], a=1 << 63, checked=True)[0] == FAULT_OVF_K   # MIN + (-1)
    assert one([MUL, 3, 0, 1 << 32], a=1 << 31, checked=True)[0] == FAULT_OVF_K
    assert one([MUL, 3, 0, 1 << 31], a=1 << 31, checked=True)[0] == APPLY
    assert one([MUL, 3, 0, U64], a=1 << 63, checked=True)[0] == FAULT_OVF_K   # MIN * (-1)
    assert one([ADD, 4, 0, 0], checked=True)[0] == FAULT_ADDR_K              # j = n
    assert one([STO, -1, 0, 0], checked=True)[0] == FAULT_ADDR_K             # j < 0
    assert one([PRI, 9, 0, 0], checked=True)[0] == FAULT_ADDR_K
    assert one([LOD, 99, 0, 0], checked=True)[0] == APPLY                    # not an address
    assert one([BNZ, 99, 0, 0], a=1, checked=True)[0] == APPLY               # jump target unchecked
    assert one([0, 0, 0, LOD], i=3, checked=True)[0] == FAULT_ADDR_K         # fetch at i = n-1
    assert one([0, 0, 0, 0], i=99, checked=True)[0] == FAULT_ADDR_K          # fetch beyond n
    assert one([0, 0, 0, 0], checked=True)[0] == FIXED                       # HLT in range
    assert one([RD, 9, 0, 0], u=(2, 1, 1), checked=True)[0] == FIXED        # RD exhausted wins
    assert one([RD, 9, 0, 0], u=(0, 1, 1), checked=True)[0] == FAULT_ADDR_K


def test_checked_fault_status_is_not_counted():
    p, po, n, t, to, caps = batch([asm((LOD, 5), (STO, 9), (LOD, 1), (ADD, 99))], [[]], 10)
    st, _ = oracle.run_packed(p, po, n, t, to, 2, 2, caps=[100], checked=True)
    assert int(st.status[0]) == oracle.FAULT_ADDR and int(st.steps[0]) == 3
    assert int(st.a[0]) == 1 and int(st.i[0]) == 6
    st, _ = oracle.run_packed(p, po, n, t, to, 2, 2, caps=[100], checked=False)
    assert int(st.status[0]) == oracle.HALTED and int(st.a[0]) == 6     # 1 + M[99 mod 10]


# ------------------------------------------------------------ closed forms
def _run(program, tape, n, ell, s=2, cap=1 << 20, w=64, budget=U64):
    p, po, nn, t, to, caps = batch([program], [tape], n, [cap])
    st, h = oracle.run_packed(p, po, nn, t, to, ell, s, caps=caps, budget=budget, w=w, hist=True)
    return st, h


def test_input_sum_closed_form():
    # loop: RD t; LOD 0; ADD t; ADD acc; STO acc; LOD 1; BNZ 0  -- halts when RD finds u_0 = l.
    # tau_h = 7 l; M[acc] = sum x mod 2^64.
    prog = asm((RD, 14), (LOD, 0), (ADD, 14), (ADD, 15), (STO, 15), (LOD, 1), (BNZ, 0))
    rng = np.random.default_rng(11)
    for ell in (0, 1, 5, 16):
        x = [int(v) for v in rng.integers(-(1 << 63), (1 << 63) - 1, size=ell, dtype=np.int64)]
        st, h = _run(prog, x, 16, ell)
        assert int(st.status[0]) == oracle.HALTED
        assert int(st.steps[0]) == 7 * ell
        assert int(st.memory(0)[15]) == sum(v & U64 for v in x) & U64
        assert int(st.u[0]) == ell
        assert list(h[1:8]) == [2 * ell, 2 * ell, 0, ell, ell, ell, 0]


def test_product_by_repeated_addition_closed_form():
    # RD A; RD B; hdr: LOD 0; ADD B; BNZ body; PRI P; HLT;
    # body: LOD 0; ADD P; ADD A; STO P; LOD -1; ADD B; STO B; LOD 1; BNZ hdr
    # tau_h = 6 + 12 x2;  y = [1, x1 x2 mod 2^64]
    prog = asm((RD, 32), (RD, 33), (LOD, 0), (ADD, 33), (BNZ, 14), (PRI, 34), (HLT, 0),
               (LOD, 0), (ADD, 34), (ADD, 32), (STO, 34), (LOD, -1), (ADD, 33), (STO, 33),
               (LOD, 1), (BNZ, 4))
    for x1, x2 in [(0, 0), (7, 0), (7, 1), (-3, 5), (1 << 62, 4), (123456789, 97)]:
        st, _ = _run(prog, [x1, x2], 40, 2)
        assert int(st.status[0]) == oracle.HALTED
        assert int(st.steps[0]) == 6 + 12 * x2
        assert [int(v) for v in st.y] == [1, (x1 * x2) & U64, 0]


def test_countdown_closed_form():
    # RD C; hdr: LOD 0; ADD C; BNZ dec; HLT; dec: LOD -1; ADD C; STO C; LOD 1; BNZ hdr
    # tau_h = 4 + 8 T
    prog = asm((RD, 20), (LOD, 0), (ADD, 20), (BNZ, 10), (HLT, 0),
               (LOD, -1), (ADD, 20), (STO, 20), (LOD, 1), (BNZ, 2))
    for T in (0, 1, 2, 17, 1000):
        st, _ = _run(prog, [T], 24, 1)
        assert int(st.status[0]) == oracle.HALTED and int(st.steps[0]) == 4 + 8 * T
        assert int(st.memory(0)[20]) == 0 and int(st.i[0]) == 8


def test_countdown_cap_boundary():
    prog = asm((RD, 20), (LOD, 0), (ADD, 20), (BNZ, 10), (HLT, 0),
               (LOD, -1), (ADD, 20), (STO, 20), (LOD, 1), (BNZ, 2))
    T = 10
    tau = 4 + 8 * T
    st, _ = _run(prog, [T], 24, 1, cap=tau)                 # tau_h == cap: the guard is evaluated
    assert int(st.status[0]) == oracle.HALTED and int(st.steps[0]) == tau
    st, _ = _run(prog, [T], 24, 1, cap=tau - 1)
    assert int(st.status[0]) == oracle.TIMEOUT and int(st.steps[0]) == tau - 1
    st, _ = _run(prog, [T], 24, 1, cap=0)
    assert int(st.status[0]) == oracle.TIMEOUT and int(st.steps[0]) == 0
    st, _ = _run(prog, [T], 24, 1, budget=37)                # budget below cap: still running
    assert int(st.status[0]) == oracle.RUNNING and int(st.steps[0]) == 37


def test_straight_line_polynomial():
    # r = x^3 + x*y + 7  (mod 2^64), evaluated by LOD/ADD/MUL/STO
    prog = asm((RD, 40), (RD, 41),
               (LOD, 0), (ADD, 40), (MUL, 40), (MUL, 40), (STO, 42),       # x^3
               (LOD, 0), (ADD, 40), (MUL, 41), (ADD, 42), (STO, 42),       # + x y
               (LOD, 7), (ADD, 42), (STO, 42), (PRI, 42), (HLT, 0))
    rng = np.random.default_rng(5)
    for _ in range(20):
        x, yv = (int(v) for v in rng.integers(-(1 << 63), (1 << 63) - 1, size=2, dtype=np.int64))
        st, _ = _run(prog, [x, yv], 44, 2)
        assert int(st.y[1]) == (x ** 3 + x * yv + 7) & U64
        assert int(st.steps[0]) == 16


# ------------------------------------------------------------ App. B
@pytest.mark.parametrize("name,tau,src", busy_beavers())
def test_busy_beaver_printed_halting_numbers(name, tau, src):
    """App. B prints tau_h for three lowered programs; they hold at w = 29."""
    low = dsl.lower(src, ell=10, s=2)
    st, _ = _run(low.words, [], max(256, low.min_mem), 10, w=29)
    assert int(st.status[0]) == oracle.HALTED
    assert int(st.steps[0]) == tau
    assert [int(v) for v in st.y] == [1, 0, 0]


@pytest.mark.parametrize("idx,formula", [(0, lambda w: 41 + 58 * (w - 3)),
                                         (1, lambda w: 12 + 45 * (w - 1)),
                                         (2, lambda w: 8 + 43 * w)])
def test_busy_beaver_closed_forms_in_w(idx, formula):
    """Hand derivation from the lowering costs: tau_h is linear in w."""
    name, tau, src = busy_beavers()[idx]
    low = dsl.lower(src, ell=10, s=2)
    assert formula(29) == tau
    for w in (8, 16, 32, 64):
        st, _ = _run(low.words, [], 256, 10, w=w)
        assert int(st.steps[0]) == formula(w)


# ------------------------------------------------------------ brute force vs spec.py
OPS = list(range(9))
ARGS = [0, 1, 2, 5, 1 << 63, U64]


def _compare_with_spec(programs, n, tape, ell, w, cap=64):
    s = 2
    p, po, nn, t, to, caps = batch(programs, [tape] * len(programs), n, cap)
    st, _ = oracle.run_packed(p, po, nn, t, to, ell, s, caps=caps, w=w)
    for v, prog in enumerate(programs):
        c0 = spec.initial(prog, tape, n, ell, s, w)
        c, steps, status = spec.run(c0, ell, s, w, cap)
        i, a, M, u, y = c
        assert int(st.steps[v]) == steps, (prog, w, n)
        assert int(st.status[v]) == status
        assert int(st.i[v]) == i and int(st.a[v]) == a
        assert [int(q) for q in st.memory(v)] == list(M)
        assert [int(q) for q in st.u[v * (ell + 1):(v + 1) * (ell + 1)]] == list(u)
        assert [int(q) for q in st.y[v * (s + 1):(v + 1) * (s + 1)]] == list(y)


@pytest.mark.parametrize("n", [6, 8])
@pytest.mark.parametrize("tape", [[], [3, -2]])
@pytest.mark.parametrize("w", [64, 8, 2])
def test_exhaustive_length_le_2_matches_spec(n, tape, w):
    instrs = [(o, a) for o in OPS for a in ARGS]
    progs = [[]] + [asm(x) for x in instrs] + [asm(x, y) for x in instrs for y in instrs]
    _compare_with_spec(progs, n, tape, 2, w)


@pytest.mark.parametrize("n,tape,w", [(6, [3, -2], 64), (8, [], 8)])
def test_exhaustive_length_3_matches_spec(n, tape, w):
    instrs = [(o, a) for o in OPS for a in ARGS]
    progs = [asm(x, y, z) for x in instrs for y in instrs for z in instrs]
    _compare_with_spec(progs, n, tape, 2, w)


def test_random_programs_match_spec():
    from paper_2604_12902_gb300.workloads import random_programs
    wl = random_programs(num_vms=96)
    st, _ = oracle.run_packed(wl.programs, wl.prog_off, wl.mem_words, wl.tapes, wl.tape_off,
                              wl.ell, wl.s, caps=wl.caps)
    for v in range(wl.num_vms):
        c0 = spec.initial([int(q) for q in wl.program_of(v)], [int(q) for q in wl.tape_of(v)],
                          int(wl.mem_words[v]), wl.ell, wl.s, 64)
        c, steps, status = spec.run(c0, wl.ell, wl.s, 64, int(wl.caps[v]))
        assert (int(st.steps[v]), int(st.status[v])) == (steps, status)
        assert [int(q) for q in st.memory(v)] == list(c[2])


# ------------------------------------------------------------ invariants
def _random_state(V=512, seed=1):
    from paper_2604_12902_gb300.workloads import random_programs
    wl = random_programs(num_vms=V, seed=seed)
    st = oracle.pack(wl.programs, wl.prog_off, wl.mem_words, wl.tapes, wl.tape_off, wl.ell, wl.s)
    return wl, st


def _same(a, b):
    for f in ("i", "a", "mem", "u", "y", "steps", "status"):
        if not np.array_equal(getattr(a, f), getattr(b, f)):
            return False
    return True


def test_resume_equals_single_run_and_halted_is_stable():
    wl, st = _random_state()
    full = st.copy()
    oracle.run(full, caps=wl.caps)
    for t1 in (0, 1, 7, 63, 200):
        part = st.copy()
        oracle.run(part, caps=wl.caps, budget=t1)
        assert np.all(part.steps <= t1)
        oracle.run(part, caps=wl.caps)
        assert _same(part, full)
    again = full.copy()
    oracle.run(again, caps=wl.caps)                                  # a stopped VM never changes
    assert _same(again, full)
    assert set(np.unique(full.status)) <= {oracle.HALTED, oracle.TIMEOUT}
    assert np.all(full.steps <= wl.caps)


def test_heads_monotone_and_single_word_writes():
    wl, st = _random_state(V=64, seed=3)
    ell, s = wl.ell, wl.s
    for v in range(wl.num_vms):
        i, a = 0, 0
        M = [int(q) for q in st.memory(v)]
        u = [int(q) for q in st.u[v * (ell + 1):(v + 1) * (ell + 1)]]
        y = [0] * (s + 1)
        for _ in range(300):
            k, i2, a2, M2, u2, y2 = oracle.step_one(64, ell, s, i, a, M, u, y)
            if k != APPLY:
                assert (i2, a2, M2, u2, y2) == (i, a, M, u, y)
                break
            assert sum(1 for p, q in zip(M, M2) if p != q) <= 1
            assert u[0] <= u2[0] <= ell and y[0] <= y2[0] <= s
            assert u2[1:] == u[1:]                                    # the tape itself is read-only
            i, a, M, u, y = i2, a2, M2, u2, y2


@pytest.mark.parametrize("w", [64, 32, 29, 5, 2])
@pytest.mark.parametrize("classic", [False, True])
def test_random_and_template_programs_match_spec_in_every_field(w, classic):
    """The C oracle and the independent spec.py transcription agree on every
    field of the final configuration for random programs (self-modifying,
    n = 64) and template programs (loops, hundreds of steps), at several word
    sizes and with both opcode sets."""
    from paper_2604_12902_gb300.workloads import random_programs, template_programs
    for wl in (random_programs(num_vms=120, seed=13 + w), template_programs(num_vms=12, seed=7 + w)):
        st, _ = oracle.run_packed(wl.programs, wl.prog_off, wl.mem_words, wl.tapes, wl.tape_off,
                                  wl.ell, wl.s, caps=wl.caps, w=w, classic=classic)
        ell, s = wl.ell, wl.s
        for v in range(wl.num_vms):
            c0 = spec.initial([int(q) for q in wl.program_of(v)], [int(q) for q in wl.tape_of(v)],
                              int(wl.mem_words[v]), ell, s, w)
            (i, a, M, u, y), steps, status = spec.run(c0, ell, s, w, int(wl.caps[v]), classic=classic)
            assert (int(st.steps[v]), int(st.status[v])) == (steps, status), (v, w, classic)
            assert (int(st.i[v]), int(st.a[v])) == (i, a)
            assert [int(q) for q in st.memory(v)] == list(M)
            assert [int(q) for q in st.u[v * (ell + 1):(v + 1) * (ell + 1)]] == list(u)
            assert [int(q) for q in st.y[v * (s + 1):(v + 1) * (s + 1)]] == list(y)
