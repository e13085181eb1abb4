"""Small helpers shared by the tests: program assembly and workload plumbing.
Nothing here computes a transition of the machine."""
from __future__ import annotations

import os

import numpy as np

LOD, ADD, MUL, STO, BNZ, RD, PRI = 1, 2, 3, 4, 5, 6, 7
HLT = 0
U64 = (1 << 64) - 1
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def asm(*instrs):
    """[(op, operand), ...] -> list of program words (operands may be negative)."""
    words = []
    for op, arg in instrs:
        words += [op, arg]
    return words


def as_i64(values):
    return np.array([((int(v) + (1 << 63)) & U64) - (1 << 63) for v in values], dtype=np.int64)


def batch(programs, tapes, n, caps=None):
    """Flat (programs, prog_off, n, tapes, tape_off, caps) for a list of programs."""
    V = len(programs)
    po = np.zeros(V + 1, np.uint64)
    po[1:] = np.cumsum([len(p) for p in programs])
    to = np.zeros(V + 1, np.uint64)
    to[1:] = np.cumsum([len(t) for t in tapes])
    flat_p = as_i64([w for p in programs for w in p])
    flat_t = as_i64([w for t in tapes for w in t])
    nn = np.array(n if hasattr(n, "__len__") else [n] * V, np.uint64)
    cc = None if caps is None else np.array(caps if hasattr(caps, "__len__") else [caps] * V, np.uint64)
    return flat_p, po, nn, flat_t, to, cc


def busy_beavers():
    """[(name, printed tau_h, source)] from tests/golden/busy_beavers.txt."""
    txt = open(os.path.join(GOLDEN, "busy_beavers.txt")).read()
    out = []
    for chunk in txt.split("\n@@ ")[1:]:
        head, body = chunk.split("\n", 1)
        name, tau = head.split()
        out.append((name, int(tau), body))
    return out
