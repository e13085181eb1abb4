"""Second, independent transcription of the word RASP (pure Python ints).

TEST INFRASTRUCTURE, for tiny exhaustive cases only. It restates Sec. 2.1 of
"Towards a Linear-Algebraic Hypervisor" with Python integers taken modulo
2^w, immutable tuples for M, u and y, and the fixed-point test written as
literal tuple equality ``step(c) == c`` (F = {c : c -> c}). It does not share
a line with ``rasp_oracle.c``: that file tests fixedness through the changed
fields; this one compares whole configurations. Wrapping semantics only (the
paper defines no faults).

Configuration: ``(i, a, M, u, y)`` with ``M`` of length n, ``u`` of length
l+1 (u[0] the read head) and ``y`` of length s+1 (y[0] the output count).

``classic=True`` takes the opcode set of the classic RASP (Sec. 1.1) on the
same words: opcode 3 is SUB, a - M_j modulo 2^w, and opcode 5 is BPA, which
jumps when a > 0 with a read as a w-bit two's complement integer.
"""
from __future__ import annotations


def initial(program, x, n: int, ell: int, s: int, w: int):
    """c_0(P, x) = <0, 0, P 0^(n-2m), x 0^(l-|x|), 0^(s+1)>  (Sec. 2.1)."""
    m2 = len(program)
    assert m2 % 2 == 0 and m2 <= n and len(x) <= ell
    mod = 1 << w
    M = tuple(int(v) % mod for v in program) + (0,) * (n - m2)
    u = (0,) + tuple(int(v) % mod for v in x) + (0,) * (ell - len(x))
    y = (0,) * (s + 1)
    return (0, 0, M, u, y)


def _set(t: tuple, k: int, v: int) -> tuple:
    """M_k <- v as the Kronecker-delta rewrite of Sec. 2.1."""
    return tuple(v if idx == k else t[idx] for idx in range(len(t)))


def step(c, ell: int, s: int, w: int, classic: bool = False):
    """The one-step transition operator of Sec. 2.1 (Sec. 1.1's opcodes 3
    and 5 with ``classic``)."""
    i, a, M, u, y = c
    mod = 1 << w
    n = len(M)
    o = M[i % n]
    j = M[((i + 1) % mod) % n]
    inc = (i + 2) % mod
    if o == 1:
        return (inc, j, M, u, y)
    if o == 2:
        return (inc, (a + M[j % n]) % mod, M, u, y)
    if o == 3 and classic:
        return (inc, (a - M[j % n]) % mod, M, u, y)
    if o == 3:
        return (inc, (a * M[j % n]) % mod, M, u, y)
    if o == 4:
        return (inc, a, _set(M, j % n, a), u, y)
    signed_a = a - mod if a >= mod // 2 else a
    jumps = (signed_a > 0) if classic else (a != 0)
    if o == 5 and jumps:
        return (j, a, M, u, y)
    if o == 5:
        return (inc, a, M, u, y)
    if o == 6 and u[0] < ell:
        bullet = u[min(u[0] + 1, ell)]
        tri = _set(u, 0, min(u[0] + 1, ell))
        return (inc, a, _set(M, j % n, bullet), tri, y)
    if o == 7:
        z = M[j % n]
        if y[0] < s:
            y2 = _set(_set(y, y[0] + 1, z), 0, y[0] + 1)
        else:
            y2 = y
        return (inc, a, M, u, y2)
    return c


def run(c, ell: int, s: int, w: int, cap: int, classic: bool = False):
    """Iterate until a fixed point or ``cap`` applied steps.
    Returns (c, steps, status) with status 1 = HALTED, 2 = TIMEOUT."""
    steps = 0
    while True:
        nxt = step(c, ell, s, w, classic)
        if nxt == c:
            return c, steps, 1
        if steps >= cap:
            return c, steps, 2
        c = nxt
        steps += 1
