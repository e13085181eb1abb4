"""Random programs of the array language, uniform by token length (Sec. 3).

The halting experiment of Sec. 3 (Fig. 1b) draws programs uniformly from the
valid code snippets of exactly L tokens of the Sec. 2.2 grammar, with a
sampler that is not available here. This module is a sampler of our own for
that distribution. For every nonterminal and every length it counts the token
strings the nonterminal derives (exact integers), then draws a derivation top
down: at each node, one alternative -- a production together with the
lengths of its parts -- with probability proportional to the number of
strings it derives. A whole program is then drawn with probability
1 / (number of valid programs of length L), up to the rounding of those
probabilities to doubles (relative error below 2^-52 per choice).

Tokens are those of the grammar: every keyword, bracket, operator and digit
is one token, so `fun f0 ( ipt : W ^ 3 ) -> W ^ 1 { scr [ 0 ] = 7 }` has 20.
A snippet is valid when its arrays fit the machine: input arity N <= l and
output arity e <= s (Sec. 2.2 reserves ipt: W^(l' <= l), opt: W^(e <= s)).
Programs whose lowering does not fit n words of memory are not valid either;
they are redrawn (from further draws of the same program's stream).

This module produces inputs only (program ASTs, their lowered words, input
tapes); it holds none of the machine's arithmetic. Randomness is
Philox4x32-10 through ``workloads.draws``: everything about program k is a
pure function of (seed, k).
"""
from __future__ import annotations

import bisect
import ctypes
from functools import lru_cache

import numpy as np

from . import dsl
from . import workloads as W

HEADER = 15            # fun f0 ( ipt : W ^ N ) -> W ^ N { ... }  without the body
REF = 4                # a [ Z ]
GET_ARRAYS = ("ipt", "scr", "opt")
PUT_ARRAYS = ("scr", "opt")


@lru_cache(maxsize=None)
def _counts(L: int):
    """Exact string counts by length 0..L for E, S and B."""
    cE = [0] * (L + 1)
    for l, c in ((1, 10), (REF, 30), (REF + 2, 600), (2 * REF + 1, 1800)):
        if l <= L:
            cE[l] = c
    cS = [0] * (L + 1)
    cB = [0] * (L + 1)
    for l in range(1, L + 1):
        s = 0
        if l - REF - 1 >= 1:
            s += 20 * cE[l - REF - 1]                                  # P = E
        if l - 9 >= 2:
            s += 30 * sum(cB[k] * cB[l - 9 - k] for k in range(1, l - 9))   # ife G { B } { B }
        if l - 7 >= 1:
            s += 30 * cB[l - 7]                                         # whl G { B }
        cS[l] = s
        b = cS[l] + (1 if l == 1 else 0)                                # S | hlt
        b += sum(cS[k] * cB[l - k - 1] for k in range(1, l - 1))       # S ; B
        cB[l] = b
    return cE, cS, cB


def count_programs(L: int, ell: int = 10, s: int = 2) -> int:
    """Number of token strings of length L derived from F with input arity
    <= min(9, l) and output arity <= min(9, s) (before the memory-fit rule)."""
    if L <= HEADER:
        return 0
    _, _, cB = _counts(L)
    return min(9, ell) * min(9, s) * cB[L - HEADER]


@lru_cache(maxsize=None)
def _table(kind: str, l: int, L: int):
    """Alternatives of nonterminal `kind` at length l: (cumulative
    probabilities, descriptors)."""
    cE, cS, cB = _counts(L)
    alts = []
    if kind == "S":
        if l - REF - 1 >= 1 and cE[l - REF - 1]:
            alts.append((20 * cE[l - REF - 1], ("put", l - REF - 1)))
        if l - 9 >= 2:
            for k in range(1, l - 9):
                w = 30 * cB[k] * cB[l - 9 - k]
                if w:
                    alts.append((w, ("ife", k, l - 9 - k)))
        if l - 7 >= 1 and cB[l - 7]:
            alts.append((30 * cB[l - 7], ("whl", l - 7)))
        total = cS[l]
    else:   # "B"
        if cS[l]:
            alts.append((cS[l], ("S",)))
        if l == 1:
            alts.append((1, ("hlt",)))
        for k in range(1, l - 1):
            w = cS[k] * cB[l - k - 1]
            if w:
                alts.append((w, ("seq", k, l - k - 1)))
        total = cB[l]
    if total == 0:
        raise ValueError("no %s of length %d" % (kind, l))
    cum, acc = [], 0
    for w, _ in alts:
        acc += w
        cum.append(acc / total)          # exact-rounded big-int division
    cum[-1] = 1.0
    return cum, [d for _, d in alts]


class _Stream:
    """Sequential uint32 draws of one program: blocks of 64 words, block b
    from stream tag (tag0 + b)."""

    def __init__(self, seed: int, pid: int, tag0: int, first_block=None):
        self.seed, self.pid, self.tag0 = seed, pid, tag0
        self.block, self.pos = 0, 0
        self.buf = first_block if first_block is not None else self._fetch(0)

    def _fetch(self, b):
        return W.draws(self.seed, self.tag0 + b, np.array([self.pid], np.uint64), 64)[0]

    def word(self) -> int:
        if self.pos == 64:
            self.block += 1
            self.buf = self._fetch(self.block)
            self.pos = 0
        w = int(self.buf[self.pos])
        self.pos += 1
        return w

    def uniform(self) -> float:
        """53-bit uniform in [0, 1)."""
        return ((self.word() >> 5) * 67108864 + (self.word() >> 6)) / 9007199254740992.0

    def below(self, k: int) -> int:
        """Integer in [0, k) by multiply-shift of one word."""
        return (self.word() * k) >> 32


class _Sampler:
    def __init__(self, L, rng: _Stream):
        self.L, self.r = L, rng

    def pick(self, kind, l):
        cum, descr = _table(kind, l, self.L)
        return descr[bisect.bisect_right(cum, self.r.uniform()) if len(cum) > 1 else 0]

    def ref(self, arrays):
        k = self.r.below(len(arrays) * 10)
        return (arrays[k // 10], k % 10)

    def expr(self, l):
        if l == 1:
            return ("const", self.r.below(10))
        if l == REF:
            return ("get", self.ref(GET_ARRAYS))
        op = "+" if self.r.below(2) == 0 else "*"
        g = ("get", self.ref(GET_ARRAYS))
        if l == REF + 2:
            return ("bin", op, g, ("const", self.r.below(10)))
        return ("bin", op, g, ("get", self.ref(GET_ARRAYS)))

    def stmt(self, l):
        d = self.pick("S", l)
        if d[0] == "put":
            return ("put", self.ref(PUT_ARRAYS), self.expr(d[1]))
        if d[0] == "ife":
            return ("ife", self.ref(GET_ARRAYS), self.block(d[1]), self.block(d[2]))
        return ("whl", self.ref(GET_ARRAYS), self.block(d[1]))

    def block(self, l):
        out = []
        while True:
            d = self.pick("B", l)
            if d[0] == "hlt":
                out.append(("hlt",))
                return out
            if d[0] == "S":
                out.append(self.stmt(l))
                return out
            out.append(self.stmt(d[1]))
            l = d[2]


def sample_fun(L: int, seed: int, pid: int, ell: int = 10, s: int = 2, attempt: int = 0,
               first_block=None, out_arity: int = 0) -> dsl.Fun:
    """The AST of program `pid` (attempt `attempt`): uniform over programs of
    exactly L tokens with input arity <= min(9, l), output arity <= min(9, s)
    (or exactly `out_arity` when it is nonzero; the arity draw is taken
    either way, so the body does not depend on it)."""
    if L <= HEADER:
        raise ValueError("L must exceed the %d header tokens" % HEADER)
    rng = _Stream(seed, pid, 0x51A0000 + 4096 * attempt, first_block if attempt == 0 else None)
    nin = 1 + rng.below(min(9, ell))
    nout = 1 + rng.below(min(9, s))
    return dsl.Fun(nin, out_arity or nout, _Sampler(L, rng).block(L - HEADER))


def fun_tokens(f: dsl.Fun) -> list:
    """Token list of an AST (inverse of dsl.parse), for checking lengths."""
    def ref(r):
        return [r[0], "[", str(r[1]), "]"]

    def expr(e):
        if e[0] == "const":
            return [str(e[1])]
        if e[0] == "get":
            return ref(e[1])
        return expr(e[2]) + [e[1]] + expr(e[3])

    def block(b):
        out = []
        for k, st in enumerate(b):
            if k:
                out.append(";")
            if st[0] == "hlt":
                out.append("hlt")
            elif st[0] == "put":
                out += ref(st[1]) + ["="] + expr(st[2])
            elif st[0] == "ife":
                out += ["ife"] + ref(st[1]) + ["{"] + block(st[2]) + ["}", "{"] + block(st[3]) + ["}"]
            else:
                out += ["whl"] + ref(st[1]) + ["{"] + block(st[2]) + ["}"]
        return out

    return (["fun", "f0", "(", "ipt", ":", "W", "^", str(f.arity), ")", "->", "W", "^", str(f.out_arity), "{"]
            + block(f.body) + ["}"])


# ---------------------------------------------------------------- C transcription
class _GenTables(ctypes.Structure):
    """gen_tables of progsampler.c: the alternatives of S and B by length."""
    _fields_ = [("L", ctypes.c_uint32),
                ("s_off", ctypes.c_void_p), ("s_cum", ctypes.c_void_p), ("s_kind", ctypes.c_void_p),
                ("s_a", ctypes.c_void_p), ("s_b", ctypes.c_void_p),
                ("b_off", ctypes.c_void_p), ("b_cum", ctypes.c_void_p), ("b_kind", ctypes.c_void_p),
                ("b_a", ctypes.c_void_p), ("b_b", ctypes.c_void_p)]


_gen_lib = None
_KIND = {"put": 0, "ife": 1, "whl": 2, "S": 0, "hlt": 1, "seq": 2}


def _gen():
    global _gen_lib
    if _gen_lib is None:
        from . import build as B
        lib = ctypes.CDLL(B.build_generator())
        P, U32, U64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        lib.gen_halting_programs.argtypes = [P, U64, U64, U64, U32, U32, U32, U32, U32, ctypes.c_int,
                                             U32, P, P, P, P, P]
        lib.gen_halting_programs.restype = ctypes.c_int
        _gen_lib = lib
    return _gen_lib


@lru_cache(maxsize=None)
def _flat_tables(L: int):
    """The alternatives tables of every length, flattened for the C sampler
    (same doubles as the Python walk uses)."""
    out = {}
    for kind, key in (("S", "s"), ("B", "b")):
        off, cum, kd, a, b = [0], [], [], [], []
        for l in range(L + 1):
            try:
                cs, ds = _table(kind, l, L)
            except ValueError:
                cs, ds = [], []
            for c, d in zip(cs, ds):
                cum.append(c)
                kd.append(_KIND[d[0]])
                a.append(d[1] if len(d) > 1 else 0)
                b.append(d[2] if len(d) > 2 else 0)
            off.append(len(cum))
        out[key] = (np.array(off, np.uint32), np.array(cum, np.float64), np.array(kd, np.int32),
                    np.array(a, np.int32), np.array(b, np.int32))
    return out


def _halting_programs_c(num_programs, L, seed, w, n, ell, s, mu, cap, first, read_inputs, out_arity):
    t = _flat_tables(L)
    keep = [t["s"], t["b"]]
    ptr = lambda x: x.ctypes.data
    T = _GenTables(L, *(ptr(x) for x in t["s"]), *(ptr(x) for x in t["b"]))
    words = np.zeros(max(num_programs * n, 1), np.int64)
    po = np.zeros(num_programs + 1, np.uint64)
    tape = np.zeros(max(num_programs * 9, 1), np.int64)
    to = np.zeros(num_programs + 1, np.uint64)
    red = np.zeros(1, np.uint64)
    rc = _gen().gen_halting_programs(ctypes.byref(T), seed, first, num_programs, ell, s, mu, n, w,
                                     1 if read_inputs else 0, out_arity, ptr(words), ptr(po), ptr(tape), ptr(to),
                                     ptr(red))
    del keep
    if rc != 0:
        raise RuntimeError("the C program sampler rejected its parameters")
    return W.Workload("halting", words[:int(po[-1])].copy(), po, np.full(num_programs, n, np.uint32),
                      tape[:int(to[-1])].copy(), to, np.full(num_programs, cap, np.uint64), ell, s, w,
                      meta=dict(L=L, seed=seed, redraws=int(red[0]), read_inputs=read_inputs,
                                out_arity=out_arity))


def halting_programs(num_programs: int, L: int = 100, seed: int = 6, w: int = 32, n: int = 250,
                     ell: int = 10, s: int = 2, mu: int = 10, cap: int = 10 ** 6,
                     first: int = 0, read_inputs: bool = False, impl: str = "c",
                     out_arity: int = 0) -> W.Workload:
    """The Sec. 3 halting workload: programs k = first .. first+count-1, each
    drawn uniformly among valid programs of L tokens and lowered by the
    Sec. 2.2 rules, on an input tape x of N uniform w-bit words. As printed,
    the Fun rule reads no input (so ipt starts at zero and x is inert, as in
    App. B); read_inputs=True prepends one RD per input word. out_arity 0
    draws the output arity e uniformly from 1..min(9, s) as the grammar
    allows; 1..min(9, s) fixes it (the program bodies stay the same). impl =
    "c" uses the C transcription (progsampler.c, the same words), "py" this
    module."""
    if not 0 <= out_arity <= min(9, s):
        raise ValueError("out_arity must be 0 (drawn) or in 1..min(9, s)")
    if impl == "c":
        return _halting_programs_c(num_programs, L, seed, w, n, ell, s, mu, cap, first, read_inputs, out_arity)
    ids = np.arange(first, first + num_programs, dtype=np.uint64)
    blocks = W.draws(seed, 0x51A0000, ids, 64)
    progs, tapes, redraws = [], [], 0
    for k, pid in enumerate(ids):
        attempt = 0
        while True:
            f = sample_fun(L, seed, int(pid), ell, s, attempt, blocks[k], out_arity)
            low = dsl.lower(f, ell=ell, s=s, mu=mu, read_inputs=read_inputs)
            if low.min_mem <= n:
                break
            attempt += 1
            redraws += 1
        progs.append(np.array([((x + (1 << 63)) % (1 << 64)) - (1 << 63) for x in low.words], np.int64))
        tapes.append(f.arity)
    tape_len = np.array(tapes, np.int64)
    tape_off = np.zeros(num_programs + 1, np.uint64)
    tape_off[1:] = np.cumsum(tape_len)
    # x uniform in F_2^(w * arity): one uniform w-bit word per input
    lo = W.draws(seed, 0x51B0000, ids, 9).astype(np.uint64)
    hi = W.draws(seed, 0x51C0000, ids, 9).astype(np.uint64) if w > 32 else np.zeros_like(lo)
    raw = ((hi << np.uint64(32)) | lo) & np.uint64((1 << w) - 1)
    tape = np.concatenate([raw[k, :tape_len[k]].view(np.int64) for k in range(num_programs)]) \
        if num_programs else np.zeros(0, np.int64)
    off = np.zeros(num_programs + 1, np.uint64)
    off[1:] = np.cumsum([len(p) for p in progs])
    flat = np.concatenate(progs) if progs else np.zeros(0, np.int64)
    return W.Workload("halting", flat, off, np.full(num_programs, n, np.uint32), tape, tape_off,
                      np.full(num_programs, cap, np.uint64), ell, s, w,
                      meta=dict(L=L, seed=seed, redraws=redraws, read_inputs=read_inputs, out_arity=out_arity))


def concat(parts) -> W.Workload:
    """One workload from consecutive chunks (e.g. generated in parallel)."""
    if len(parts) == 1:
        return parts[0]
    def offs(lens):
        o = np.zeros(len(lens) + 1, np.uint64)
        o[1:] = np.cumsum(lens)
        return o
    plen = np.concatenate([p.prog_off[1:] - p.prog_off[:-1] for p in parts])
    tlen = np.concatenate([p.tape_off[1:] - p.tape_off[:-1] for p in parts])
    p0 = parts[0]
    meta = dict(p0.meta)
    meta["redraws"] = sum(p.meta.get("redraws", 0) for p in parts)
    return W.Workload(p0.name, np.concatenate([p.programs for p in parts]), offs(plen),
                      np.concatenate([p.mem_words for p in parts]), np.concatenate([p.tapes for p in parts]),
                      offs(tlen), np.concatenate([p.caps for p in parts]), p0.ell, p0.s, p0.w, meta=meta)


def _chunk_job(a):
    return halting_programs(**a)


def halting_programs_parallel(num_programs: int, workers: int = 1, chunk: int = 1 << 15, **kw) -> W.Workload:
    """halting_programs chunk by chunk on `workers` threads (the C sampler runs
    without the interpreter lock) or, for impl="py", spawned processes;
    identical to one call, since every program is a function of (seed, k)."""
    first = kw.pop("first", 0)
    jobs = [dict(kw, num_programs=min(chunk, num_programs - o), first=first + o)
            for o in range(0, num_programs, chunk)]
    if workers <= 1 or len(jobs) == 1:
        return concat([_chunk_job(j) for j in jobs])
    if kw.get("impl", "c") == "c":
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(workers) as ex:
            return concat(list(ex.map(_chunk_job, jobs)))
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        return concat(pool.map(_chunk_job, jobs))
