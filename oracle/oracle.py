"""CPU oracle for the word RASP -- Python wrapper around ``rasp_oracle.c``.

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module. The product path (the
``paper_2604_12902_gb300`` package) never imports it, and this module imports
nothing from the product.

The C file is the plain serial statement of the machine of Sec. 2.1 of
"Towards a Linear-Algebraic Hypervisor" (configuration space, c_0, the case
equation, fixed-point halting); this wrapper only builds it with gcc and
marshals numpy arrays. Every array is laid out the way the paper writes the
configuration: ``u`` holds l+1 words per VM (u[0] = read head) and ``y`` holds
s+1 words per VM (y[0] = output count).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rasp_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "librasp_oracle.so")

RUNNING, HALTED, TIMEOUT, FAULT_OVERFLOW, FAULT_ADDR = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "RUNNING", 1: "HALTED", 2: "TIMEOUT", 3: "FAULT_OVERFLOW", 4: "FAULT_ADDR"}
U64_MAX = (1 << 64) - 1

_lock = threading.Lock()
_lib = None


class _Params(ctypes.Structure):
    _fields_ = [("w", ctypes.c_uint32), ("checked", ctypes.c_uint32),
                ("ell", ctypes.c_uint64), ("s", ctypes.c_uint64),
                ("isa", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


ISA_WORD, ISA_CLASSIC = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2) into oracle/_build."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                               "-Wall", "-Wextra", "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.ro_pack.argtypes = [ctypes.POINTER(_Params), ctypes.c_uint64] + [P] * 13
            lib.ro_pack.restype = ctypes.c_int
            lib.ro_run.argtypes = ([ctypes.POINTER(_Params), ctypes.c_uint64, ctypes.c_uint64]
                                   + [P] * 10 + [ctypes.c_uint64, P])
            lib.ro_run.restype = ctypes.c_int
            lib.ro_step_one.argtypes = [ctypes.POINTER(_Params)] + [P] * 3 + [ctypes.c_uint64, P, P]
            lib.ro_step_one.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(arr: np.ndarray):
    assert arr.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(arr.ctypes.data)


def _u64(x) -> np.ndarray:
    """int64 two's-complement or uint64 input -> contiguous uint64 (same bits)."""
    if isinstance(x, (list, tuple)):
        return np.array([int(v) & U64_MAX for v in x], dtype=np.uint64)
    a = np.asarray(x)
    if a.dtype == np.uint64:
        return np.ascontiguousarray(a)
    if a.dtype == np.int64:
        return np.ascontiguousarray(a).view(np.uint64)
    if a.dtype == object or a.size == 0:
        return np.array([int(v) & U64_MAX for v in a.ravel()], dtype=np.uint64).reshape(a.shape)
    return np.ascontiguousarray(a.astype(np.int64)).view(np.uint64)


class State:
    """Configurations of a batch of machines, in the paper's layout."""

    def __init__(self, w, checked, ell, s, n, mem_off, mem, i, a, u, y, steps, status, classic=False):
        self.w, self.checked, self.ell, self.s = int(w), bool(checked), int(ell), int(s)
        self.classic = bool(classic)
        self.n, self.mem_off, self.mem = n, mem_off, mem
        self.i, self.a, self.u, self.y = i, a, u, y
        self.steps, self.status = steps, status

    @property
    def count(self) -> int:
        return int(self.n.shape[0])

    def params(self) -> _Params:
        return _Params(self.w, 1 if self.checked else 0, self.ell, self.s,
                       ISA_CLASSIC if self.classic else ISA_WORD, 0)

    def memory(self, v: int) -> np.ndarray:
        o = int(self.mem_off[v])
        return self.mem[o:o + int(self.n[v])]

    def copy(self) -> "State":
        return State(self.w, self.checked, self.ell, self.s, self.n.copy(), self.mem_off.copy(),
                     self.mem.copy(), self.i.copy(), self.a.copy(), self.u.copy(),
                     self.y.copy(), self.steps.copy(), self.status.copy(), self.classic)


def pack(programs, prog_off, n, tapes, tape_off, ell: int, s: int,
         w: int = 64, checked: bool = False, classic: bool = False) -> State:
    """c_0(P, x) for every VM (Sec. 2.1). ``programs``/``tapes`` are flat word
    arrays with ``*_off`` prefix offsets (length V+1); ``n`` is per-VM memory.
    ``classic`` selects the classic opcode set (Sec. 1.1: SUB, BPA)."""
    lib = _load()
    n = _u64(n)
    V = n.shape[0]
    mem_off = np.zeros(V, dtype=np.uint64)
    if V:
        mem_off[1:] = np.cumsum(n[:-1], dtype=np.uint64)
    total = int(n.sum()) if V else 0
    mem = np.zeros(max(total, 1), dtype=np.uint64)
    prog = _u64(programs) if len(programs) else np.zeros(1, np.uint64)
    tape = _u64(tapes) if len(tapes) else np.zeros(1, np.uint64)
    po, to = _u64(prog_off), _u64(tape_off)
    st = State(w, checked, ell, s, n, mem_off, mem,
               np.zeros(V, np.uint64), np.zeros(V, np.uint64),
               np.zeros(max(V * (ell + 1), 1), np.uint64), np.zeros(max(V * (s + 1), 1), np.uint64),
               np.zeros(V, np.uint64), np.zeros(V, np.uint8), classic)
    p = st.params()
    rc = lib.ro_pack(ctypes.byref(p), V, _ptr(n), _ptr(mem_off), _ptr(mem), _ptr(prog), _ptr(po),
                     _ptr(tape), _ptr(to), _ptr(st.i), _ptr(st.a), _ptr(st.u), _ptr(st.y),
                     _ptr(st.steps), _ptr(st.status))
    if rc != 0:
        raise ValueError("oracle pack rejected the batch (odd program, 2m > n, n = 0 or |x| > l)")
    return st


def run(st: State, caps=None, budget: int = U64_MAX, hist: bool = False,
        threads: int = 1, first: int = 0, count: int | None = None):
    """Advance VMs [first, first+count) in place; returns the 9-entry opcode
    histogram when ``hist`` (index 1..7 = opcode, 8 = PRI on a full tape,
    0 = taken BNZ)."""
    lib = _load()
    V = st.count
    if count is None:
        count = V - first
    cap = np.full(V, U64_MAX, np.uint64) if caps is None else _u64(caps)
    assert cap.shape[0] == V
    p = st.params()
    hists = []

    def work(lo, hi):
        h = np.zeros(9, np.uint64)
        rc = lib.ro_run(ctypes.byref(p), lo, hi - lo, _ptr(st.n), _ptr(st.mem_off), _ptr(st.mem),
                        _ptr(st.i), _ptr(st.a), _ptr(st.u), _ptr(st.y), _ptr(st.steps), _ptr(cap),
                        _ptr(st.status), int(budget) & U64_MAX, _ptr(h) if hist else None)
        if rc != 0:
            raise ValueError("oracle run rejected its parameters")
        hists.append(h)

    if threads <= 1 or count < 2 * threads:
        work(first, first + count)
    else:
        bounds = np.linspace(first, first + count, 4 * threads + 1).astype(np.int64)
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda k: work(int(bounds[k]), int(bounds[k + 1])), range(len(bounds) - 1)))
    if hist:
        return np.sum(hists, axis=0).astype(np.uint64)
    return None


def step_one(w: int, ell: int, s: int, i: int, a: int, M, u, y, checked: bool = False,
             classic: bool = False):
    """One transition of one machine. Returns (kind, i, a, M, u, y) with kind
    0 = applied, 1 = fixed point, 2 = address fault, 3 = overflow fault."""
    lib = _load()
    p = _Params(w, 1 if checked else 0, ell, s, ISA_CLASSIC if classic else ISA_WORD, 0)
    ii = np.array([i & U64_MAX], np.uint64)
    aa = np.array([a & U64_MAX], np.uint64)
    MM, uu, yy = _u64(list(M)).copy(), _u64(list(u)).copy(), _u64(list(y)).copy()
    assert uu.shape[0] == ell + 1 and yy.shape[0] == s + 1
    kind = lib.ro_step_one(ctypes.byref(p), _ptr(ii), _ptr(aa), _ptr(MM), MM.shape[0], _ptr(uu), _ptr(yy))
    return kind, int(ii[0]), int(aa[0]), [int(v) for v in MM], [int(v) for v in uu], [int(v) for v in yy]


def run_packed(programs, prog_off, n, tapes, tape_off, ell, s, caps=None, budget=U64_MAX,
               w=64, checked=False, hist=False, threads=1, classic=False):
    """pack + run in one call; returns (State, hist or None)."""
    st = pack(programs, prog_off, n, tapes, tape_off, ell, s, w=w, checked=checked, classic=classic)
    h = run(st, caps=caps, budget=budget, hist=hist, threads=threads)
    return st, h
