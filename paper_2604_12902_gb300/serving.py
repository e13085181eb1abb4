"""Serving loop over the pool calls of ``include/rasp.h`` (continuous batching).

``Pool`` is the thin binding (argument marshalling only). ``poisson_run``
drives it open-loop: requests arrive at exponential inter-arrival times,
are submitted when they arrive, and are polled until done; a finished
request is read back (which frees its device memory and admits waiting
requests). Latency is measured from arrival to the first pass that sees the
request done; throughput is the VM-steps of all finished requests over the
wall time of the run.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import rasp as R

QUEUED, RUNNING, DONE = 0, 1, 2


class rasp_request(ctypes.Structure):
    _fields_ = [("words", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("num_programs", ctypes.c_uint64),
                ("prog_of_vm", ctypes.c_void_p), ("tape", ctypes.c_void_p), ("tape_off", ctypes.c_void_p),
                ("caps", ctypes.c_void_p), ("mem_words", ctypes.c_void_p), ("num_vms", ctypes.c_uint64),
                ("max_steps", ctypes.c_uint64)]


class rasp_pool_counters(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint64) for name in ("admitted", "completed", "kernel_launches", "kernel_returns",
                                                     "ring_published", "vms_in_flight", "kernel_ctas")]


_typed = False


def _lib():
    global _typed
    L = R.lib()
    if not _typed:
        P, U64 = ctypes.c_void_p, ctypes.c_uint64
        L.rasp_pool_create.argtypes = [ctypes.POINTER(R.rasp_config), U64, ctypes.POINTER(ctypes.c_void_p)]
        L.rasp_pool_submit.argtypes = [P, ctypes.POINTER(rasp_request), ctypes.POINTER(U64)]
        L.rasp_pool_poll.argtypes = [P, U64, ctypes.POINTER(ctypes.c_int)]
        L.rasp_pool_read.argtypes = [P, U64, ctypes.POINTER(R.rasp_state_view)]
        L.rasp_pool_info.argtypes = [P, ctypes.POINTER(U64), ctypes.POINTER(U64), ctypes.POINTER(U64)]
        L.rasp_pool_cancel.argtypes = [P, U64]
        L.rasp_pool_next_done.argtypes = [P, ctypes.POINTER(U64)]
        L.rasp_pool_stats.argtypes = [P, ctypes.POINTER(rasp_pool_counters)]
        L.rasp_pool_destroy.argtypes = [P]
        L.rasp_pool_destroy.restype = None
        L.rasp_pool_last_error.restype = ctypes.c_char_p
        for name in ("rasp_pool_create", "rasp_pool_submit", "rasp_pool_poll", "rasp_pool_read", "rasp_pool_info",
                     "rasp_pool_cancel", "rasp_pool_next_done", "rasp_pool_stats"):
            getattr(L, name).restype = ctypes.c_int
        _typed = True
    return L


def _check(rc):
    if rc != 0:
        raise R.RaspError(rc, _lib().rasp_pool_last_error().decode())


class Pool:
    """A device arena serving many requests (each one batch of VMs)."""

    def __init__(self, arena_bytes: int, in_cap: int, out_cap: int, word_bits: int = 64,
                 semantics: int = R.WRAP, flags: int = 0):
        self.s = int(out_cap)
        cfg = R.rasp_config(word_bits, semantics, in_cap, out_cap, flags, 0, 0, 0, 0, 0, None, None, 0)
        h = ctypes.c_void_p()
        _check(_lib().rasp_pool_create(ctypes.byref(cfg), int(arena_bytes), ctypes.byref(h)))
        self.h = h
        self.meta = {}

    def submit(self, wl, max_steps: int = R.U64_MAX) -> int:
        arrs = dict(words=np.ascontiguousarray(wl.programs, np.int64) if len(wl.programs) else np.zeros(1, np.int64),
                    offsets=np.ascontiguousarray(wl.prog_off, np.uint64),
                    pvm=None if wl.prog_of_vm is None else np.ascontiguousarray(wl.prog_of_vm, np.uint32),
                    tape=np.ascontiguousarray(wl.tapes, np.int64) if len(wl.tapes) else np.zeros(1, np.int64),
                    toff=np.ascontiguousarray(wl.tape_off, np.uint64),
                    caps=np.ascontiguousarray(wl.caps, np.uint64),
                    mem=np.ascontiguousarray(wl.mem_words, np.uint32))
        q = rasp_request(R._p(arrs["words"]), R._p(arrs["offsets"]), arrs["offsets"].shape[0] - 1,
                         R._p(arrs["pvm"]), R._p(arrs["tape"]), R._p(arrs["toff"]), R._p(arrs["caps"]),
                         R._p(arrs["mem"]), wl.num_vms, int(max_steps) & R.U64_MAX)
        t = ctypes.c_uint64(0)
        _check(_lib().rasp_pool_submit(self.h, ctypes.byref(q), ctypes.byref(t)))
        self.meta[t.value] = (wl.num_vms, wl.mem_words)
        return t.value

    def poll(self, ticket: int) -> int:
        st = ctypes.c_int(0)
        _check(_lib().rasp_pool_poll(self.h, ticket, ctypes.byref(st)))
        return st.value

    def read(self, ticket: int, mem: bool = False) -> dict:
        V, mw = self.meta.pop(ticket)
        out = dict(i=np.empty(V, np.int64), a=np.empty(V, np.int64), steps=np.empty(V, np.uint64),
                   status=np.empty(V, np.uint8), uhead=np.empty(V, np.uint32), ylen=np.empty(V, np.uint32),
                   y=np.empty((V, self.s), np.int64))
        nw = int(np.asarray(mw, np.uint64).sum()) if mem else 0
        if mem:
            out["mem"] = np.empty(nw, np.int64)
        v = R.rasp_state_view(R._p(out["i"]), R._p(out["a"]), R._p(out["steps"]), R._p(out["status"]),
                              R._p(out["uhead"]), R._p(out["ylen"]), R._p(out["y"]) if self.s else None,
                              R._p(out["mem"]) if mem else None, nw)
        _check(_lib().rasp_pool_read(self.h, ticket, ctypes.byref(v)))
        return out

    def next_done(self) -> int:
        """A finished request not handed out before, or 0 (non-blocking)."""
        t = ctypes.c_uint64(0)
        _check(_lib().rasp_pool_next_done(self.h, ctypes.byref(t)))
        return t.value

    def cancel(self, ticket: int):
        """Withdraw a request still waiting for admission."""
        _check(_lib().rasp_pool_cancel(self.h, ticket))
        self.meta.pop(ticket, None)

    def info(self) -> dict:
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(_lib().rasp_pool_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return dict(in_use=a.value, waiting=b.value, running=c.value)

    def stats(self) -> dict:
        """Pool counters: requests admitted and completed, serving kernel
        instances launched and returned, VMs published and in flight."""
        st = rasp_pool_counters()
        _check(_lib().rasp_pool_stats(self.h, ctypes.byref(st)))
        return {name: int(getattr(st, name)) for name, _ in rasp_pool_counters._fields_}

    def close(self):
        if getattr(self, "h", None):
            _lib().rasp_pool_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def poisson_run(pool: Pool, requests, lam: float, duration: float, seed: int = 0, max_steps: int = R.U64_MAX,
                poll_interval: float = 2e-4, keep_results: bool = False, max_waiting: int | None = None):
    """Open-loop Poisson arrivals (rate `lam` per second) for `duration`
    seconds, cycling through the pre-built `requests` (workloads); then drain.
    With `max_waiting`, an arrival that finds that many requests waiting for
    admission is rejected (admission control: an overloaded pool would
    otherwise hold an ever-growing backlog of request copies). Returns a dict
    with per-request latencies (s), VM-steps, throughput and rejections."""
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    next_arrival = t0 + rng.exponential(1.0 / lam)
    inflight = {}                      # ticket -> (arrival time, request index)
    lat, steps, sizes, results = [], 0, [], []
    k = rejected = 0
    while True:
        now = time.perf_counter()
        while now >= next_arrival and next_arrival - t0 < duration:
            idx = k % len(requests)
            if max_waiting is not None and pool.info()["waiting"] >= max_waiting:
                rejected += 1
            else:
                tk = pool.submit(requests[idx], max_steps)
                inflight[tk] = (next_arrival, idx)
            k += 1
            next_arrival += rng.exponential(1.0 / lam)
        while True:                          # every request that finished since the last pass
            tk = pool.next_done()
            if not tk:
                break
            t_done = time.perf_counter()
            arr, idx = inflight.pop(tk)
            res = pool.read(tk)
            lat.append(t_done - arr)
            steps += int(res["steps"].sum())
            sizes.append(requests[idx].num_vms)
            if keep_results:
                results.append((idx, res))
        if next_arrival - t0 >= duration and not inflight:
            break
        time.sleep(poll_interval)
    wall = time.perf_counter() - t0
    lat = np.array(lat)
    return dict(requests=len(lat), rejected=rejected, wall_s=wall, vm_steps=steps, vm_steps_per_s=steps / wall,
                p50_ms=float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
                p99_ms=float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
                mean_vms=float(np.mean(sizes)) if sizes else 0.0, results=results, latencies=lat)
