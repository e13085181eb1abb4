"""Property test: the C oracle and the independent spec.py transcription agree
in every field on machines drawn by hypothesis -- any word size 1..64, both
opcode sets, memories from one word, empty tapes and zero output capacity,
operands near n, near 2^w and negative, and step caps from 0."""
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from oracle import oracle, spec  # noqa: E402
from tests.helpers import batch  # noqa: E402


@st.composite
def machines(draw):
    w = draw(st.sampled_from([1, 2, 3, 7, 8, 16, 29, 32, 63, 64]))
    n = draw(st.integers(1, 40))
    m = draw(st.integers(min(1, n // 2), n // 2))
    big = (1 << w) - 1
    operand = st.one_of(st.integers(-3, n + 3), st.sampled_from([big, big - 1, 1 << (w - 1), -(1 << 63)]),
                        st.integers(-(1 << 63), (1 << 63) - 1))
    prog = []
    for _ in range(m):
        # mostly the seven defined opcodes, one time in ten an invalid one (a fixed point)
        op = draw(st.integers(1, 7)) if draw(st.integers(0, 9)) else draw(st.sampled_from([-1, 0, 8, 9]))
        prog += [op, draw(operand)]
    ell = draw(st.integers(0, 4))
    tape = [draw(st.integers(-(1 << 63), (1 << 63) - 1)) for _ in range(draw(st.integers(0, ell)))]
    s = draw(st.integers(0, 3))
    cap = draw(st.integers(0, 300))
    classic = draw(st.booleans())
    return w, n, prog, ell, tape, s, cap, classic


@settings(max_examples=1000, deadline=None, derandomize=True)
@given(machines())
def test_c_oracle_equals_spec(mc):
    w, n, prog, ell, tape, s, cap, classic = mc
    p, po, nn, t, to, caps = batch([prog], [tape], n, cap)
    got, _ = oracle.run_packed(p, po, nn, t, to, ell, s, caps=caps, w=w, classic=classic)
    c0 = spec.initial(prog, tape, n, ell, s, w)
    (i, a, M, u, y), steps, status = spec.run(c0, ell, s, w, cap, classic=classic)
    assert (int(got.steps[0]), int(got.status[0])) == (steps, status)
    assert (int(got.i[0]), int(got.a[0])) == (i, a)
    assert [int(q) for q in got.memory(0)] == list(M)
    assert [int(q) for q in got.u[:ell + 1]] == list(u)
    assert [int(q) for q in got.y[:s + 1]] == list(y)
