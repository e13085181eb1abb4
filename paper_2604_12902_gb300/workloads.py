"""Seeded synthetic workloads for the batched word RASP.

This module produces *inputs* only -- program words, input tapes, memory
sizes and step caps -- and holds none of the machine's arithmetic. Both the
CUDA path and the CPU oracle consume what it returns.

Randomness comes from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11), implemented here from that
definition with numpy uint32/uint64 arithmetic. Every drawn word is a pure
function of (seed, stream tag, VM id, index), so any subset of VMs can be
regenerated on its own and chunked generation equals whole generation.

Instruction words follow the machine's encoding (Sec. 2.1): instruction k of
a program occupies words 2k (opcode) and 2k+1 (operand), opcodes 1 LOD,
2 ADD, 3 MUL, 4 STO, 5 BNZ, 6 RD, 7 PRI, and "0 0" is the halting pair of
Sec. 2.2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LOD, ADD, MUL, STO, BNZ, RD, PRI = 1, 2, 3, 4, 5, 6, 7
U64_MAX = (1 << 64) - 1

# Philox4x32 constants (Salmon et al. 2011, Table 2 / Random123).
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint32(0x9E3779B9)
_PHILOX_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32(c0, c1, c2, c3, k0, k1, rounds: int = 10):
    """Philox4x32-R block function on uint32 arrays (broadcasting)."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint32) for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint32)
    k1 = np.asarray(k1, dtype=np.uint32)
    with np.errstate(over="ignore"):
        for r in range(rounds):
            if r:
                k0 = (k0 + _PHILOX_W0).astype(np.uint32)
                k1 = (k1 + _PHILOX_W1).astype(np.uint32)
            p0 = c0.astype(np.uint64) * _PHILOX_M0
            p1 = c2.astype(np.uint64) * _PHILOX_M1
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK32).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def draws(seed: int, tag: int, vm_ids: np.ndarray, count: int) -> np.ndarray:
    """uint32 matrix [len(vm_ids), count]; entry (v, k) depends only on
    (seed, tag, vm_ids[v], k). Counter = (k // 4, vm_lo, vm_hi, tag),
    key = (seed_lo, seed_hi); lane k % 4 of the Philox output."""
    vm = np.asarray(vm_ids, dtype=np.uint64).reshape(-1, 1)
    blocks = (count + 3) // 4
    b = np.arange(blocks, dtype=np.uint32).reshape(1, -1)
    vlo = (vm & _MASK32).astype(np.uint32)
    vhi = (vm >> np.uint64(32)).astype(np.uint32)
    t = np.uint32(tag & 0xFFFFFFFF)
    k0 = np.uint32(seed & 0xFFFFFFFF)
    k1 = np.uint32((seed >> 32) & 0xFFFFFFFF)
    out = philox4x32(np.broadcast_to(b, (vm.shape[0], blocks)), vlo, vhi, t, k0, k1)
    m = np.stack(out, axis=-1).reshape(vm.shape[0], blocks * 4)
    return np.ascontiguousarray(m[:, :count])


def uniform_int(u32: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """Map uint32 draws to integers in [lo, hi] by multiply-shift
    (floor(u * span / 2^32)); bias < span / 2^32."""
    span = hi - lo + 1
    assert 1 <= span <= (1 << 32)
    r = (u32.astype(np.uint64) * np.uint64(span)) >> np.uint64(32)
    return r.astype(np.int64) + lo


def log_uniform_int(u32: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """Integers log-uniform on [lo, hi]: floor(lo * ((hi+1)/lo)^U), U in (0,1).
    Uses float64 exp/log, so a value that lands on an integer boundary may
    differ between libm builds; inputs of one run are always shared by both
    sides, so parity never depends on it."""
    uu = (u32.astype(np.float64) + 0.5) / 4294967296.0
    x = np.floor(lo * np.exp(uu * (math.log(hi + 1) - math.log(lo))))
    return np.clip(x, lo, hi).astype(np.int64)


@dataclass
class Workload:
    """A batch of machines ready for ``rasp_load_programs``/``rasp_load_inputs``
    and for the oracle. Words are int64 two's complement."""
    name: str
    programs: np.ndarray           # int64, flat
    prog_off: np.ndarray           # uint64, V+1 (or P+1 with prog_of_vm)
    mem_words: np.ndarray          # uint32, V   (n per VM)
    tapes: np.ndarray              # int64, flat
    tape_off: np.ndarray           # uint64, V+1
    caps: np.ndarray               # uint64, V
    ell: int                       # input tape capacity l
    s: int                         # output capacity s
    w: int = 64
    prog_of_vm: np.ndarray | None = None   # uint32, V: shared-program index
    meta: dict = field(default_factory=dict)

    @property
    def num_vms(self) -> int:
        return int(self.mem_words.shape[0])

    def program_of(self, v: int) -> np.ndarray:
        p = int(self.prog_of_vm[v]) if self.prog_of_vm is not None else v
        return self.programs[int(self.prog_off[p]):int(self.prog_off[p + 1])]

    def tape_of(self, v: int) -> np.ndarray:
        return self.tapes[int(self.tape_off[v]):int(self.tape_off[v + 1])]

    def expanded_programs(self):
        """(programs, prog_off) with one program per VM (resolves prog_of_vm)."""
        if self.prog_of_vm is None:
            return self.programs, self.prog_off
        lens = (self.prog_off[1:] - self.prog_off[:-1])[self.prog_of_vm]
        off = np.zeros(self.num_vms + 1, np.uint64)
        off[1:] = np.cumsum(lens, dtype=np.uint64)
        parts = [self.program_of(v) for v in range(self.num_vms)]
        flat = np.concatenate(parts) if parts else np.zeros(0, np.int64)
        return flat, off

    def subset(self, ids) -> "Workload":
        """The workload restricted to VMs ``ids`` (programs expanded)."""
        ids = np.asarray(ids, dtype=np.int64)
        progs = [self.program_of(int(v)) for v in ids]
        tapes = [self.tape_of(int(v)) for v in ids]
        return Workload(self.name + "[subset]", _flat(progs), _offsets(progs),
                        self.mem_words[ids].copy(), _flat(tapes), _offsets(tapes),
                        self.caps[ids].copy(), self.ell, self.s, self.w, None, dict(self.meta))


def _flat(parts):
    return np.concatenate(parts).astype(np.int64) if parts and sum(len(p) for p in parts) else np.zeros(0, np.int64)


def _offsets(parts):
    off = np.zeros(len(parts) + 1, np.uint64)
    off[1:] = np.cumsum([len(p) for p in parts], dtype=np.uint64)
    return off


def _regular_offsets(count: int, length: int) -> np.ndarray:
    return (np.arange(count + 1, dtype=np.uint64) * np.uint64(length))


# ---------------------------------------------------------------------------
# Random programs: 32 instructions, opcodes uniform over 1..7, operands
# uniform in [0, 63], 64-word memory (the program fills it), tape of 4 ints
# uniform in [-100, 100], step cap 256.
# ---------------------------------------------------------------------------
def random_programs(num_vms: int = 1024, seed: int = 1, instructions: int = 32,
                    mem_words: int = 64, tape_len: int = 4, tape_lo: int = -100,
                    tape_hi: int = 100, operand_hi: int = 63, cap: int = 256,
                    s: int = 8, opcode_lo: int = 1, opcode_hi: int = 7,
                    first_vm: int = 0) -> Workload:
    ids = np.arange(first_vm, first_vm + num_vms, dtype=np.uint64)
    ops = uniform_int(draws(seed, 1, ids, instructions), opcode_lo, opcode_hi)
    arg = uniform_int(draws(seed, 2, ids, instructions), 0, operand_hi)
    prog = np.empty((num_vms, 2 * instructions), np.int64)
    prog[:, 0::2] = ops
    prog[:, 1::2] = arg
    tape = uniform_int(draws(seed, 3, ids, tape_len), tape_lo, tape_hi)
    return Workload("random", prog.reshape(-1), _regular_offsets(num_vms, 2 * instructions),
                    np.full(num_vms, mem_words, np.uint32), tape.reshape(-1),
                    _regular_offsets(num_vms, tape_len), np.full(num_vms, cap, np.uint64),
                    ell=tape_len, s=s, meta=dict(seed=seed, instructions=instructions))


# ---------------------------------------------------------------------------
# Template programs (straight-line arithmetic blocks plus 1..3 sequential
# counter-bounded loops, trip counts uniform in [1, 64]).
#
# Memory (n words): code in [0, 2*I), inputs in [D, D+T), loop counters in
# [D+T, D+T+3), scratch above. D = 2*I.
# Program = RD prologue (one RD per input word) | S_0 | loop_1 | S_1 | ... |
#           loop_L | S_L | PRI x2 | 0 0, exactly I instructions.
# loop_k (12 + b_k instructions, counter c, trip T):
#     LOD T; STO c;
#   hdr: LOD 0; ADD c; BNZ body; LOD 1; BNZ exit;
#   body: <b_k straight-line instructions>; LOD -1; ADD c; STO c; LOD 1; BNZ hdr;
#   exit:
# A straight-line instruction is LOD k (k in [-8, 8]), ADD d / MUL d (d any
# data word) or STO d (d a scratch word), uniformly.
# ---------------------------------------------------------------------------
_SEG_PROLOGUE, _SEG_FILL, _SEG_LOOP, _SEG_EPI = 0, 1, 2, 3


def template_programs(num_vms: int = 1 << 20, seed: int = 2, instructions: int = 64,
                      mem_words: int = 256, tape_len: int = 16, tape_lo: int = -1000,
                      tape_hi: int = 1000, cap: int = 4096, s: int = 8,
                      trip_lo: int = 1, trip_hi: int = 64, loops_lo: int = 1,
                      loops_hi: int = 3, body_lo: int = 1, body_hi: int = 3,
                      p_nonhalting: float = 0.0, first_vm: int = 0,
                      chunk: int = 1 << 16) -> Workload:
    I = instructions
    assert mem_words >= 2 * I + tape_len + 3 + 8, "memory too small for the template"
    progs = np.empty((num_vms, 2 * I), np.int64)
    tapes = np.empty((num_vms, tape_len), np.int64)
    for c0 in range(0, num_vms, chunk):
        cnt = min(chunk, num_vms - c0)
        ids = np.arange(first_vm + c0, first_vm + c0 + cnt, dtype=np.uint64)
        progs[c0:c0 + cnt] = _template_chunk(ids, seed, I, mem_words, tape_len, trip_lo, trip_hi,
                                             loops_lo, loops_hi, body_lo, body_hi, p_nonhalting)
        tapes[c0:c0 + cnt] = uniform_int(draws(seed, 4, ids, tape_len), tape_lo, tape_hi)
    return Workload("templates", progs.reshape(-1), _regular_offsets(num_vms, 2 * I),
                    np.full(num_vms, mem_words, np.uint32), tapes.reshape(-1),
                    _regular_offsets(num_vms, tape_len), np.full(num_vms, cap, np.uint64),
                    ell=tape_len, s=s, meta=dict(seed=seed, instructions=I))


def _template_chunk(ids, seed, I, n, T, trip_lo, trip_hi, loops_lo, loops_hi,
                    body_lo, body_hi, p_nonhalting):
    V = ids.shape[0]
    D = 2 * I
    counters = D + T
    scratch_lo = D + T + 3
    st = draws(seed, 1, ids, 12)
    L = uniform_int(st[:, 0], loops_lo, loops_hi)                       # loops per program
    trips = uniform_int(st[:, 1:4], trip_lo, trip_hi)                   # [V,3]
    body = uniform_int(st[:, 4:7], body_lo, body_hi)                    # [V,3]
    present = np.arange(3)[None, :] < L[:, None]
    loop_len = np.where(present, 12 + body, 0)
    fixed = T + 3                                                       # prologue + PRI PRI HLT
    fill_total = I - fixed - loop_len.sum(axis=1)
    if np.any(fill_total < 0):
        raise ValueError("template does not fit in %d instructions" % I)
    # split the filler over the L+1 gaps: gap g < L takes U[0, rest // 2], the last takes the rest
    fills = np.zeros((V, 4), np.int64)
    rest = fill_total.copy()
    for g in range(3):
        take = uniform_int(st[:, 7 + g], 0, 1 << 20) % (rest // 2 + 1)
        take = np.where(g < L, take, 0)
        fills[:, g] = take
        rest = rest - take
    fills[np.arange(V), L] += rest
    # the decrement of loop k is dropped (making the VM non-halting) with probability p_nonhalting
    nonhalt = (st[:, 10].astype(np.float64) / 4294967296.0) < p_nonhalting
    # segment lengths in order: prologue, fill0, loop1, fill1, loop2, fill2, loop3, fill3, epilogue
    seg_len = np.stack([np.full(V, T), fills[:, 0], loop_len[:, 0], fills[:, 1], loop_len[:, 1],
                        fills[:, 2], loop_len[:, 2], fills[:, 3], np.full(V, 3)], axis=1)
    seg_kind = np.array([_SEG_PROLOGUE, _SEG_FILL, _SEG_LOOP, _SEG_FILL, _SEG_LOOP,
                         _SEG_FILL, _SEG_LOOP, _SEG_FILL, _SEG_EPI])
    seg_loop = np.array([-1, -1, 0, -1, 1, -1, 2, -1, -1])
    seg_end = np.cumsum(seg_len, axis=1)
    assert np.all(seg_end[:, -1] == I)
    seg_start = seg_end - seg_len
    t = np.arange(I)[None, :]
    seg = (t[:, :, None] >= seg_end[:, None, :]).sum(axis=2)              # [V,I] segment index
    start = np.take_along_axis(seg_start, seg, axis=1)
    r = t - start                                                         # offset in segment
    kind = seg_kind[seg]
    li = np.clip(seg_loop[seg], 0, 2)
    b = np.take_along_axis(body, li, axis=1)
    T_k = np.take_along_axis(trips, li, axis=1)
    c_k = counters + li
    # random straight-line instructions (fill and loop bodies)
    cls = uniform_int(draws(seed, 2, ids, I), 0, 3)
    oper = draws(seed, 3, ids, I)
    rnd_op = np.array([LOD, ADD, MUL, STO])[cls]
    rnd_arg = np.where(cls == 0, uniform_int(oper, -8, 8),
                       np.where(cls == 3, uniform_int(oper, scratch_lo, n - 1),
                                uniform_int(oper, D, n - 1)))
    op = np.zeros((V, I), np.int64)
    arg = np.zeros((V, I), np.int64)
    # prologue: RD D + r
    m = kind == _SEG_PROLOGUE
    op[m] = RD
    arg[m] = (D + r)[m]
    m = kind == _SEG_FILL
    op[m] = rnd_op[m]
    arg[m] = rnd_arg[m]
    # epilogue: PRI d, PRI d, 0 0
    m = (kind == _SEG_EPI) & (r < 2)
    op[m] = PRI
    arg[m] = uniform_int(oper, D, n - 1)[m]
    # loops
    drop = nonhalt[:, None]
    lp = kind == _SEG_LOOP
    table = [
        (r == 0, LOD, T_k), (r == 1, STO, c_k), (r == 2, LOD, 0), (r == 3, ADD, c_k),
        (r == 4, BNZ, 2 * (start + 7)), (r == 5, LOD, 1), (r == 6, BNZ, 2 * (start + 12 + b)),
        (r == 7 + b, LOD, np.where(drop, 0, -1)), (r == 8 + b, ADD, c_k), (r == 9 + b, STO, c_k),
        (r == 10 + b, LOD, 1), (r == 11 + b, BNZ, 2 * (start + 2)),
    ]
    for cond, o, a in table:
        mm = lp & cond
        op[mm] = o
        arg[mm] = np.broadcast_to(a, (V, I))[mm]
    mb = lp & (r >= 7) & (r < 7 + b)
    op[mb] = rnd_op[mb]
    arg[mb] = rnd_arg[mb]
    out = np.empty((V, 2 * I), np.int64)
    out[:, 0::2] = op
    out[:, 1::2] = arg
    return out



def draws_ragged(seed: int, tag: int, vm_ids: np.ndarray, counts: np.ndarray) -> np.ndarray:
    """Flat uint32 draws: the first counts[v] entries of draws(seed, tag,
    [vm_ids[v]], .) for every v, concatenated (same values as `draws`)."""
    vm = np.asarray(vm_ids, dtype=np.uint64)
    counts = np.asarray(counts, dtype=np.int64)
    nblk = (counts + 3) // 4
    bvm = np.repeat(np.arange(vm.shape[0]), nblk)
    bstart = np.concatenate([[0], np.cumsum(nblk)[:-1]])
    bidx = (np.arange(bvm.shape[0]) - bstart[bvm]).astype(np.uint32)
    v64 = vm[bvm]
    out = philox4x32(bidx, (v64 & _MASK32).astype(np.uint32), (v64 >> np.uint64(32)).astype(np.uint32),
                     np.uint32(tag & 0xFFFFFFFF), np.uint32(seed & 0xFFFFFFFF),
                     np.uint32((seed >> 32) & 0xFFFFFFFF))
    blocks = np.stack(out, axis=-1).reshape(-1)                 # 4 words per block, in block order
    svm = np.repeat(np.arange(vm.shape[0]), counts)
    sstart = np.concatenate([[0], np.cumsum(counts)[:-1]])
    t = np.arange(svm.shape[0]) - sstart[svm]
    return blocks[4 * bstart[svm] + t]


def _uniform_rows(u32: np.ndarray, lo, hi) -> np.ndarray:
    """uniform_int with per-element bounds."""
    span = (np.asarray(hi, np.int64) - np.asarray(lo, np.int64) + 1).astype(np.uint64)
    return ((u32.astype(np.uint64) * span) >> np.uint64(32)).astype(np.int64) + lo


# ---------------------------------------------------------------------------
# Uneven batch: program length log-uniform in [8, 512] instructions, memory
# log-uniform in [16, 4096] words (raised to fit the program and its data,
# never rounded), step cap log-uniform in [64, 65536]. Programs follow the
# template structure scaled to their length: R = min(l, (I-3)//4) RD
# instructions, up to three counter-bounded loops (as many as fit), straight-
# line blocks, PRI PRI HLT. With probability p_nonhalting the loop decrement
# is LOD 0 instead of LOD -1, so a program with a loop never halts.
# ---------------------------------------------------------------------------
def uneven_programs(num_vms: int = 1 << 22, seed: int = 3, len_lo: int = 8, len_hi: int = 512,
                    n_lo: int = 16, n_hi: int = 4096, cap_lo: int = 64, cap_hi: int = 65536,
                    p_nonhalting: float = 0.15, tape_len: int = 16, s: int = 8, first_vm: int = 0,
                    chunk: int = 1 << 16, workers: int = 0) -> Workload:
    """``workers`` > 1 generates chunks in a spawn-context process pool (safe
    after CUDA has been initialised in the calling process); the result does
    not depend on it."""
    args = [(first_vm + c0, min(chunk, num_vms - c0), seed, len_lo, len_hi, n_lo, n_hi, cap_lo, cap_hi,
             p_nonhalting, tape_len) for c0 in range(0, num_vms, chunk)]
    if workers > 1 and len(args) > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(min(workers, len(args)), mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_uneven_job, args))
    else:
        parts = [_uneven_job(a) for a in args]
    progs, offs, mems, tapes, caps = [], [], [], [], []
    total = 0
    for words, I, n, cap, tape in parts:
        progs.append(words)
        offs.append(total + np.concatenate([[0], np.cumsum(2 * I)[:-1]]))
        total += int(2 * I.sum())
        mems.append(n)
        caps.append(cap)
        tapes.append(tape)
    prog_off = np.zeros(num_vms + 1, np.uint64)
    prog_off[:-1] = np.concatenate(offs).astype(np.uint64)
    prog_off[-1] = total
    return Workload("uneven", np.concatenate(progs), prog_off, np.concatenate(mems).astype(np.uint32),
                    np.concatenate(tapes).reshape(-1), _regular_offsets(num_vms, tape_len),
                    np.concatenate(caps).astype(np.uint64), ell=tape_len, s=s,
                    meta=dict(seed=seed, p_nonhalting=p_nonhalting))


def _uneven_job(a):
    first, cnt, seed, len_lo, len_hi, n_lo, n_hi, cap_lo, cap_hi, p_nonhalting, tape_len = a
    ids = np.arange(first, first + cnt, dtype=np.uint64)
    words, I, n, cap = _uneven_chunk(ids, seed, len_lo, len_hi, n_lo, n_hi, cap_lo, cap_hi,
                                     p_nonhalting, tape_len)
    tape = uniform_int(draws(seed, 4, ids, tape_len), -1000, 1000)
    return words, I, n, cap, tape


def _uneven_chunk(ids, seed, len_lo, len_hi, n_lo, n_hi, cap_lo, cap_hi, p_nonhalting, tape_len):
    V = ids.shape[0]
    st = draws(seed, 1, ids, 16)
    I = log_uniform_int(st[:, 0], len_lo, len_hi)
    R = np.minimum(tape_len, np.maximum(0, (I - 3) // 4))
    D = 2 * I
    n = np.maximum(log_uniform_int(st[:, 1], n_lo, n_hi), D + R + 3 + 8)
    cap = log_uniform_int(st[:, 2], cap_lo, cap_hi)
    nonhalt = (st[:, 3].astype(np.float64) / 4294967296.0) < p_nonhalting
    lmax = np.clip((I - R - 3) // 13, 0, 3)
    L = np.where(lmax > 0, _uniform_rows(st[:, 4], np.minimum(1, lmax), lmax), 0)
    trips = np.stack([uniform_int(st[:, 5 + k], 1, 64) for k in range(3)], axis=1)
    extra = np.maximum(0, I - R - 3 - 13 * L) // np.maximum(L, 1)
    body = np.stack([1 + np.minimum(uniform_int(st[:, 8 + k], 0, 2), extra) for k in range(3)], axis=1)
    present = np.arange(3)[None, :] < L[:, None]
    loop_len = np.where(present, 12 + body, 0)
    fill_total = I - R - 3 - loop_len.sum(axis=1)
    assert np.all(fill_total >= 0)
    fills = np.zeros((V, 4), np.int64)
    rest = fill_total.copy()
    for g in range(3):
        take = uniform_int(st[:, 11 + g], 0, 1 << 20) % (rest // 2 + 1)
        take = np.where(g < L, take, 0)
        fills[:, g] = take
        rest = rest - take
    fills[np.arange(V), L] += rest
    seg_len = np.stack([R, fills[:, 0], loop_len[:, 0], fills[:, 1], loop_len[:, 1],
                        fills[:, 2], loop_len[:, 2], fills[:, 3], np.full(V, 3)], axis=1)
    seg_kind = np.array([_SEG_PROLOGUE, _SEG_FILL, _SEG_LOOP, _SEG_FILL, _SEG_LOOP,
                         _SEG_FILL, _SEG_LOOP, _SEG_FILL, _SEG_EPI])
    seg_loop = np.array([-1, -1, 0, -1, 1, -1, 2, -1, -1])
    seg_end = np.cumsum(seg_len, axis=1)
    assert np.all(seg_end[:, -1] == I)
    # flat per-instruction arrays
    vm = np.repeat(np.arange(V), I)
    start = np.concatenate([[0], np.cumsum(I)[:-1]])
    t = np.arange(vm.shape[0]) - start[vm]
    bounds = (start[:, None] + seg_end).reshape(-1)
    g = np.searchsorted(bounds, np.arange(vm.shape[0]), side="right")
    k = g % 9
    seg_start = (seg_end - seg_len)[vm, k]
    r = t - seg_start
    kind = seg_kind[k]
    li = np.clip(seg_loop[k], 0, 2)
    b = body[vm, li]
    Tk = trips[vm, li]
    Dv, Rv, nv = D[vm], R[vm], n[vm]
    c_k = Dv + Rv + li
    scratch_lo = Dv + Rv + 3
    cls = uniform_int(draws_ragged(seed, 2, ids, I), 0, 3)
    oper = draws_ragged(seed, 3, ids, I)
    rnd_op = np.array([LOD, ADD, MUL, STO])[cls]
    rnd_arg = np.where(cls == 0, uniform_int(oper, -8, 8),
                       np.where(cls == 3, _uniform_rows(oper, scratch_lo, nv - 1),
                                _uniform_rows(oper, Dv, nv - 1)))
    op = np.zeros(vm.shape[0], np.int64)
    arg = np.zeros(vm.shape[0], np.int64)
    m = kind == _SEG_PROLOGUE
    op[m] = RD
    arg[m] = (Dv + r)[m]
    m = kind == _SEG_FILL
    op[m] = rnd_op[m]
    arg[m] = rnd_arg[m]
    m = (kind == _SEG_EPI) & (r < 2)
    op[m] = PRI
    arg[m] = _uniform_rows(oper, Dv, nv - 1)[m]
    drop = nonhalt[vm]
    lp = kind == _SEG_LOOP
    st0 = start[vm] * 0 + seg_start
    table = [
        (r == 0, LOD, Tk), (r == 1, STO, c_k), (r == 2, LOD, 0), (r == 3, ADD, c_k),
        (r == 4, BNZ, 2 * (st0 + 7)), (r == 5, LOD, 1), (r == 6, BNZ, 2 * (st0 + 12 + b)),
        (r == 7 + b, LOD, np.where(drop, 0, -1)), (r == 8 + b, ADD, c_k), (r == 9 + b, STO, c_k),
        (r == 10 + b, LOD, 1), (r == 11 + b, BNZ, 2 * (st0 + 2)),
    ]
    for cond, o, a in table:
        mm = lp & cond
        op[mm] = o
        arg[mm] = np.broadcast_to(a, vm.shape)[mm]
    mb = lp & (r >= 7) & (r < 7 + b)
    op[mb] = rnd_op[mb]
    arg[mb] = rnd_arg[mb]
    words = np.empty(2 * vm.shape[0], np.int64)
    words[0::2] = op
    words[1::2] = arg
    return words, I, n, cap


# ---------------------------------------------------------------------------
# Shared-program rollout: P candidate programs (length 48, the loop templates
# above with at most two loops) each run on R input tapes of 8 ints uniform
# in [-50, 50]; memory = 96 program words + 128 private data words (n = 224);
# step cap 2048. VM v runs program v // R.
# ---------------------------------------------------------------------------
def shared_programs(num_programs: int = 16384, vms_per_program: int = 256, seed: int = 4,
                    instructions: int = 48, data_words: int = 128, tape_len: int = 8,
                    tape_lo: int = -50, tape_hi: int = 50, cap: int = 2048, s: int = 8) -> Workload:
    n = 2 * instructions + data_words
    base = template_programs(num_vms=num_programs, seed=seed, instructions=instructions, mem_words=n,
                             tape_len=tape_len, loops_hi=2)
    V = num_programs * vms_per_program
    ids = np.arange(V, dtype=np.uint64)
    tape = uniform_int(draws(seed, 9, ids, tape_len), tape_lo, tape_hi)
    return Workload("shared", base.programs, base.prog_off, np.full(V, n, np.uint32), tape.reshape(-1),
                    _regular_offsets(V, tape_len), np.full(V, cap, np.uint64), ell=tape_len, s=s,
                    prog_of_vm=np.repeat(np.arange(num_programs, dtype=np.uint32), vms_per_program),
                    meta=dict(seed=seed, programs=num_programs, vms_per_program=vms_per_program))
