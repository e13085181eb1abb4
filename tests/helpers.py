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


# ------------------------------------------------------------------ parity plumbing
def oracle_state(wl, budget=U64, checked=False, hist=False, threads=1, classic=False):
    """Run a workload through the CPU oracle (programs expanded per VM);
    ``classic`` selects the classic opcode set (SUB, BPA)."""
    from oracle import oracle
    progs, po = wl.expanded_programs()
    return oracle.run_packed(progs, po, wl.mem_words, wl.tapes, wl.tape_off, wl.ell, wl.s,
                             caps=wl.caps, budget=budget, w=wl.w, checked=checked, hist=hist,
                             threads=threads, classic=classic)


def assert_same_state(got, st, ell, s, ids=None, what=""):
    """GPU state (library layout, optionally only VMs `ids`) == oracle state."""
    V = st.count
    sel = slice(None) if ids is None else ids
    u64 = lambda x: np.asarray(x).view(np.uint64) if np.asarray(x).dtype == np.int64 else np.asarray(x)
    for key, want in (("i", st.i), ("a", st.a), ("steps", st.steps), ("status", st.status),
                      ("uhead", st.u[0::ell + 1][:V]), ("ylen", st.y[0::s + 1][:V])):
        g = u64(got[key])[sel]
        w = np.asarray(want)
        if not np.array_equal(g.astype(np.uint64), w.astype(np.uint64)):
            bad = np.nonzero(g.astype(np.uint64) != w.astype(np.uint64))[0]
            raise AssertionError("%s: field %s differs at %d VMs, first %d: gpu %r oracle %r"
                                 % (what, key, bad.size, bad[0], g[bad[0]], w[bad[0]]))
    if s:
        gy = u64(got["y"])[sel].reshape(V, s)
        wy = st.y.reshape(V, s + 1)[:, 1:]
        assert np.array_equal(gy, wy), "%s: outputs y differ" % what
    if "mem" in got and ids is None:
        gm = u64(got["mem"])
        if not np.array_equal(gm, st.mem[:gm.shape[0]]):
            bad = np.nonzero(gm != st.mem[:gm.shape[0]])[0]
            raise AssertionError("%s: memory differs at %d words, first word %d" % (what, bad.size, bad[0]))


def checked_workload(V=4096, seed=11):
    """Random programs whose operands straddle [0, n) and whose data are large,
    so that address and overflow faults both occur under CHECKED semantics
    (n = 48, 20 instructions, 4 RDs of values near +-2^63 first, cap 500)."""
    from paper_2604_12902_gb300 import workloads as W
    ids = np.arange(V, dtype=np.uint64)
    n = 48
    ops = np.array([1, 2, 2, 2, 3, 3, 3, 4, 5, 7, 0, 8])[W.uniform_int(W.draws(seed, 1, ids, 20), 0, 11)]
    arg = W.uniform_int(W.draws(seed, 2, ids, 20), 30, n + 3)
    arg[:, ::5] -= 36                                           # some negative operands
    ops[:, :4] = RD                                             # read the large inputs first
    arg[:, :4] = np.arange(40, 44)
    prog = np.empty((V, 40), np.int64)
    prog[:, 0::2] = ops
    prog[:, 1::2] = arg
    big = W.uniform_int(W.draws(seed, 3, ids, 4), -(1 << 31), (1 << 31) - 1).astype(np.int64)
    tape = big * np.int64(1 << 32)
    return W.Workload("checked", prog.reshape(-1), np.arange(V + 1, dtype=np.uint64) * 40,
                      np.full(V, n, np.uint32), tape.reshape(-1), np.arange(V + 1, dtype=np.uint64) * 4,
                      np.full(V, 500, np.uint64), 4, 3)
