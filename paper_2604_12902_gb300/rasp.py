"""Thin ctypes binding of ``include/rasp.h`` (argument marshalling only).

Every function of the C ABI is exposed under the same name; ``Batch`` wraps
one ``rasp_batch`` with numpy in/out. Device memory for a batch comes from
PyTorch (a ``torch.uint8`` CUDA tensor passed to the library as its arena)
and work is ordered on the current torch CUDA stream, so torch's allocator
and stream semantics apply. All computation happens in the library's CUDA
kernels; if the library has not been built this module raises instead of
falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

RASP_OK, RASP_EINVAL, RASP_ENOMEM, RASP_ECUDA, RASP_ESTATE, RASP_EDEVICE = 0, -1, -2, -3, -4, -5
RUNNING, HALTED, TIMEOUT, FAULT_OVERFLOW, FAULT_ADDR = 0, 1, 2, 3, 4
WRAP, CHECKED = 0, 1
SCHED_AUTO, SCHED_PLAIN, SCHED_PERSIST, SCHED_PERSIST_GL, SCHED_SHARED = 0x00, 0x10, 0x20, 0x30, 0x40
DISPATCH_SELECT, DISPATCH_VOTE = 0x000, 0x100
COLLECT_STATS = 0x1000
ISA_CLASSIC = 0x8000
BUDGET_ROUNDS = 0x10000
STEP_BLOCK = 0x20000
SHARED_PROGRAM = 0x2000
CUDA_GRAPH = 0x4000
U64_MAX = (1 << 64) - 1


class rasp_config(ctypes.Structure):
    _fields_ = [("word_bits", ctypes.c_uint32), ("semantics", ctypes.c_uint32),
                ("in_cap", ctypes.c_uint32), ("out_cap", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("epoch", ctypes.c_uint32),
                ("warps_per_cta", ctypes.c_uint32), ("refill_min", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("stream", ctypes.c_void_p), ("arena", ctypes.c_void_p),
                ("arena_bytes", ctypes.c_uint64)]


class rasp_state_view(ctypes.Structure):
    _fields_ = [("i", ctypes.c_void_p), ("a", ctypes.c_void_p), ("steps", ctypes.c_void_p),
                ("status", ctypes.c_void_p), ("uhead", ctypes.c_void_p), ("ylen", ctypes.c_void_p),
                ("y", ctypes.c_void_p), ("mem", ctypes.c_void_p), ("mem_words", ctypes.c_uint64)]


class rasp_stats(ctypes.Structure):
    _fields_ = [("vm_steps", ctypes.c_uint64), ("running", ctypes.c_uint64),
                ("halted", ctypes.c_uint64), ("timeout", ctypes.c_uint64),
                ("fault_overflow", ctypes.c_uint64), ("fault_addr", ctypes.c_uint64),
                ("op_steps", ctypes.c_uint64 * 8), ("pri_full", ctypes.c_uint64),
                ("bnz_taken", ctypes.c_uint64), ("launches", ctypes.c_uint64)]


class RaspError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("rasp error %d: %s" % (code, msg))
        self.code = code


_lib = None
EXPORTS = ["rasp_batch_bytes", "rasp_batch_create", "rasp_load_programs", "rasp_load_inputs",
           "rasp_reset", "rasp_run", "rasp_sync", "rasp_read_state", "rasp_load_state",
           "rasp_read_stats", "rasp_describe", "rasp_autotune", "rasp_halting_histogram",
           "rasp_top_halting", "rasp_plan_bucket", "rasp_load_programs_i32", "rasp_batch_destroy",
           "rasp_last_error", "rasp_version"]


def lib():
    """The loaded C library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError("librasp_gb300.so is not built (%s); run __graft_entry__.build()" % LIB)
        L = ctypes.CDLL(LIB)
        P, U64, U32, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        cfgp = ctypes.POINTER(rasp_config)
        L.rasp_batch_bytes.argtypes = [cfgp, U64, P, ctypes.POINTER(U64)]
        L.rasp_batch_create.argtypes = [cfgp, U64, P, ctypes.POINTER(ctypes.c_void_p)]
        L.rasp_load_programs.argtypes = [P, P, P, U64, P]
        L.rasp_load_inputs.argtypes = [P, P, P, P]
        L.rasp_reset.argtypes = [P]
        L.rasp_run.argtypes = [P, U64]
        L.rasp_sync.argtypes = [P]
        L.rasp_read_state.argtypes = [P, U64, U64, ctypes.POINTER(rasp_state_view)]
        L.rasp_load_state.argtypes = [P, U64, U64, ctypes.POINTER(rasp_state_view)]
        L.rasp_read_stats.argtypes = [P, ctypes.POINTER(rasp_stats)]
        L.rasp_describe.argtypes = [P, ctypes.c_char_p, U64]
        L.rasp_autotune.argtypes = [P, U64, U32]
        L.rasp_halting_histogram.argtypes = [P, P, U32, P, P]
        L.rasp_top_halting.argtypes = [P, U32, P, P, P]
        L.rasp_plan_bucket.argtypes = [P, U32, U32, U32, U32, U32]
        L.rasp_load_programs_i32.argtypes = [P, P, P, U64, P]
        L.rasp_batch_destroy.argtypes = [P]
        L.rasp_batch_destroy.restype = None
        L.rasp_last_error.restype = ctypes.c_char_p
        L.rasp_version.restype = ctypes.c_char_p
        for name in EXPORTS[:16]:
            getattr(L, name).restype = I
        _lib = L
    return _lib


def _check(rc):
    if rc != RASP_OK:
        raise RaspError(rc, lib().rasp_last_error().decode())
    return rc


def _p(arr):
    return None if arr is None else ctypes.c_void_p(arr.ctypes.data)


def _c(arr, dtype):
    return np.ascontiguousarray(arr, dtype=dtype) if arr is not None else None


# ---- same-name wrappers of the C ABI (raise RaspError on failure) ----------
def rasp_batch_bytes(cfg: rasp_config, mem_words: np.ndarray) -> int:
    mw = _c(mem_words, np.uint32)
    out = ctypes.c_uint64(0)
    _check(lib().rasp_batch_bytes(ctypes.byref(cfg), mw.shape[0], _p(mw), ctypes.byref(out)))
    return out.value


def rasp_batch_create(cfg: rasp_config, mem_words: np.ndarray):
    mw = _c(mem_words, np.uint32)
    h = ctypes.c_void_p()
    _check(lib().rasp_batch_create(ctypes.byref(cfg), mw.shape[0], _p(mw), ctypes.byref(h)))
    return h


def rasp_load_programs(h, words, offsets, prog_of_vm=None):
    w = _c(words, np.int64) if len(words) else np.zeros(1, np.int64)
    o = _c(offsets, np.uint64)
    pv = _c(prog_of_vm, np.uint32)
    _check(lib().rasp_load_programs(h, _p(w), _p(o), o.shape[0] - 1, _p(pv)))


def rasp_load_programs_i32(h, words, offsets, prog_of_vm=None):
    """Programs as int32 words (each stands for its sign-extended int64)."""
    w = _c(words, np.int32) if len(words) else np.zeros(1, np.int32)
    o = _c(offsets, np.uint64)
    pv = _c(prog_of_vm, np.uint32)
    _check(lib().rasp_load_programs_i32(h, _p(w), _p(o), o.shape[0] - 1, _p(pv)))


def rasp_load_inputs(h, tape, offsets, caps=None):
    t = _c(tape, np.int64) if len(tape) else np.zeros(1, np.int64)
    o = _c(offsets, np.uint64)
    c = _c(caps, np.uint64)
    _check(lib().rasp_load_inputs(h, _p(t), _p(o), _p(c)))


def rasp_reset(h):
    _check(lib().rasp_reset(h))


def rasp_run(h, max_steps: int = U64_MAX):
    _check(lib().rasp_run(h, int(max_steps) & U64_MAX))


def rasp_sync(h):
    _check(lib().rasp_sync(h))


def rasp_read_state(h, first: int, count: int, view: rasp_state_view):
    _check(lib().rasp_read_state(h, first, count, ctypes.byref(view)))


def rasp_load_state(h, first: int, count: int, view: rasp_state_view):
    _check(lib().rasp_load_state(h, first, count, ctypes.byref(view)))


def rasp_read_stats(h) -> rasp_stats:
    st = rasp_stats()
    _check(lib().rasp_read_stats(h, ctypes.byref(st)))
    return st


def rasp_describe(h) -> dict:
    import json
    buf = ctypes.create_string_buffer(1 << 14)
    _check(lib().rasp_describe(h, buf, len(buf)))
    return json.loads(buf.value.decode())


def rasp_autotune(h, max_steps: int = U64_MAX, reps: int = 2):
    _check(lib().rasp_autotune(h, int(max_steps) & U64_MAX, reps))


def rasp_plan_bucket(h, bucket: int, sched: int, epoch: int = 0, warps_per_cta: int = 0, ctas_per_sm: int = 0):
    _check(lib().rasp_plan_bucket(h, bucket, sched, epoch, warps_per_cta, ctas_per_sm))


def rasp_halting_histogram(h, edges, counts, other=None):
    """Device histogram of tau_h over HALTED VMs; counts[k] for
    edges[k] <= steps < edges[k+1] (uint64 arrays); other[4] optional."""
    return _check(lib().rasp_halting_histogram(h, _p(edges), len(edges) - 1, _p(counts), _p(other)))


def rasp_top_halting(h, k: int):
    """(tau_h, vm) of the k HALTED VMs with the largest tau_h, best first
    (ties: smaller VM index), selected on the device."""
    st = np.zeros(k, np.uint64)
    vm = np.zeros(k, np.uint32)
    found = np.zeros(1, np.uint32)
    _check(lib().rasp_top_halting(h, int(k), _p(st), _p(vm), _p(found)))
    n = int(found[0])
    return st[:n], vm[:n]


def rasp_batch_destroy(h):
    lib().rasp_batch_destroy(h)


def rasp_last_error() -> str:
    return lib().rasp_last_error().decode()


def rasp_version() -> str:
    return lib().rasp_version().decode()


def _torch_stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Batch:
    """One batch of machines. Arrays use the library layout: ``y`` is
    [count, s] (y_1..y_s), ``uhead``/``ylen`` are u_0/y_0, ``mem`` is the
    concatenation of each VM's n words."""

    def __init__(self, mem_words, in_cap: int, out_cap: int, word_bits: int = 64,
                 semantics: int = WRAP, flags: int = 0, epoch: int = 0, stream=None,
                 torch_arena: bool = True, warps_per_cta: int = 0, refill_min: int = 0,
                 ctas_per_sm: int = 0):
        import torch
        self.mem_words = np.ascontiguousarray(mem_words, dtype=np.uint32)
        self.V = int(self.mem_words.shape[0])
        self.ell, self.s, self.w = int(in_cap), int(out_cap), int(word_bits)
        self.cfg = rasp_config(word_bits, semantics, in_cap, out_cap, flags, epoch, warps_per_cta,
                               refill_min, ctas_per_sm, 0,
                               stream if stream is not None else _torch_stream(), None, 0)
        self._arena = None
        if torch_arena:
            nbytes = rasp_batch_bytes(self.cfg, self.mem_words)
            self._arena = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            self.cfg.arena = ctypes.c_void_p(self._arena.data_ptr())
            self.cfg.arena_bytes = nbytes
        self.h = rasp_batch_create(self.cfg, self.mem_words)
        self.n_total = int(self.mem_words.astype(np.uint64).sum())

    # loads -------------------------------------------------------------
    def load_programs(self, words, offsets, prog_of_vm=None):
        rasp_load_programs(self.h, words, offsets, prog_of_vm)

    def load_inputs(self, tape, offsets, caps=None):
        rasp_load_inputs(self.h, tape, offsets, caps)

    def load_workload(self, wl):
        """Load a ``workloads.Workload`` (programs, tapes, caps)."""
        self.load_programs(wl.programs, wl.prog_off, wl.prog_of_vm)
        self.load_inputs(wl.tapes, wl.tape_off, wl.caps)

    def reset(self):
        rasp_reset(self.h)

    def run(self, max_steps: int = U64_MAX):
        rasp_run(self.h, max_steps)

    def sync(self):
        rasp_sync(self.h)

    def read_state(self, first: int = 0, count: int | None = None, mem: bool = True) -> dict:
        if count is None:
            count = self.V - first
        out = dict(i=np.empty(count, np.int64), a=np.empty(count, np.int64),
                   steps=np.empty(count, np.uint64), status=np.empty(count, np.uint8),
                   uhead=np.empty(count, np.uint32), ylen=np.empty(count, np.uint32),
                   y=np.empty((count, self.s), np.int64))
        nw = int(self.mem_words[first:first + count].astype(np.uint64).sum()) if mem else 0
        if mem:
            out["mem"] = np.empty(nw, np.int64)
        v = rasp_state_view(_p(out["i"]), _p(out["a"]), _p(out["steps"]), _p(out["status"]),
                            _p(out["uhead"]), _p(out["ylen"]), _p(out["y"]) if self.s else None,
                            _p(out["mem"]) if mem else None, nw)
        rasp_read_state(self.h, first, count, v)
        return out

    def load_state(self, st: dict, first: int = 0):
        count = int(st["i"].shape[0])
        arrs = {k: None for k in ("i", "a", "steps", "status", "uhead", "ylen", "y", "mem")}
        dt = dict(i=np.int64, a=np.int64, steps=np.uint64, status=np.uint8, uhead=np.uint32,
                  ylen=np.uint32, y=np.int64, mem=np.int64)
        for k in arrs:
            if st.get(k) is not None:
                arrs[k] = np.ascontiguousarray(st[k], dtype=dt[k])
        nw = int(arrs["mem"].shape[0]) if arrs["mem"] is not None else 0
        v = rasp_state_view(*(_p(arrs[k]) for k in ("i", "a", "steps", "status", "uhead", "ylen", "y", "mem")), nw)
        rasp_load_state(self.h, first, count, v)

    def stats(self) -> dict:
        st = rasp_read_stats(self.h)
        return dict(vm_steps=st.vm_steps, running=st.running, halted=st.halted, timeout=st.timeout,
                    fault_overflow=st.fault_overflow, fault_addr=st.fault_addr,
                    op_steps=[st.op_steps[k] for k in range(8)], pri_full=st.pri_full,
                    bnz_taken=st.bnz_taken, launches=st.launches)

    def describe(self) -> dict:
        return rasp_describe(self.h)

    def top_halting(self, k: int):
        """(tau_h, vm) of the k HALTED VMs with the largest tau_h, best first."""
        return rasp_top_halting(self.h, k)

    def halting_histogram(self, edges):
        """(counts per bin, other) of the halting times: counts[k] = HALTED VMs
        with edges[k] <= steps < edges[k+1]; other = [running, timeout,
        faulted, halted outside the edges]."""
        e = np.ascontiguousarray(edges, dtype=np.uint64)
        counts = np.zeros(len(e) - 1, np.uint64)
        other = np.zeros(4, np.uint64)
        rasp_halting_histogram(self.h, e, counts, other)
        return counts, other

    def plan_bucket(self, bucket: int, sched: int, epoch: int = 0, warps_per_cta: int = 0, ctas_per_sm: int = 0):
        """Pin the schedule of memory-size bucket ``bucket`` (its "index" in
        ``describe()["buckets"]``)."""
        rasp_plan_bucket(self.h, bucket, sched, epoch, warps_per_cta, ctas_per_sm)

    def autotune(self, max_steps: int = U64_MAX, reps: int = 2) -> dict:
        """Time the candidate schedules on this batch (state unchanged) and
        keep the fastest; returns the trial report."""
        rasp_autotune(self.h, max_steps, reps)
        return self.describe()["autotune"]

    def close(self):
        if getattr(self, "h", None):
            rasp_batch_destroy(self.h)
            self.h = None
        self._arena = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- rasp_run_static: a caller-owned state store, no allocation ----------
class rasp_static_run(ctypes.Structure):
    _fields_ = [("i", ctypes.c_void_p), ("a", ctypes.c_void_p), ("steps", ctypes.c_void_p),
                ("cap", ctypes.c_void_p), ("status", ctypes.c_void_p), ("uhead", ctypes.c_void_p),
                ("ylen", ctypes.c_void_p), ("n", ctypes.c_void_p), ("mem_off", ctypes.c_void_p),
                ("mem", ctypes.c_void_p), ("tape", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("num_vms", ctypes.c_uint64), ("word_bits", ctypes.c_uint32),
                ("semantics", ctypes.c_uint32), ("in_cap", ctypes.c_uint32), ("out_cap", ctypes.c_uint32),
                ("max_steps", ctypes.c_uint64), ("stream", ctypes.c_void_p), ("err_buf", ctypes.c_char_p),
                ("err_buf_size", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("mem_words", ctypes.c_uint64), ("rejected", ctypes.c_void_p)]


RASP_STATIC_MAX_VMS = 1 << 20


def rasp_run_static(run: rasp_static_run) -> int:
    """Call rasp_run_static; returns its status code (0 = OK). The error
    message, if any, is written to run.err_buf."""
    L = lib()
    if not getattr(L.rasp_run_static, "_typed", False):
        L.rasp_run_static.argtypes = [ctypes.POINTER(rasp_static_run)]
        L.rasp_run_static.restype = ctypes.c_int
        L.rasp_run_static._typed = True
    return L.rasp_run_static(ctypes.byref(run))
