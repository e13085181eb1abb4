"""Generate -> run -> filter: a search over random programs.

The paper's stated use of the batched machine is search over program space
(busy beavers, superoptimisation; Sec. 3 and Sec. 5). Here round r draws
programs r*B .. (r+1)*B - 1 uniformly among the valid programs of L tokens
(``sampler.py``), runs them on the device to tau_max, and keeps, across
rounds, the k halting programs with the largest tau_h -- the longest-running
programs that still halt, i.e. busy-beaver candidates for L tokens. The
filter runs on the device (``rasp_top_halting``); only k (tau_h, id) pairs per
round come back. Generating round r+1 on the host (the C sampler on a thread
pool) overlaps the device run of round r.

Ties in tau_h go to the smaller program id, so the result is a function of
(L, seed, rounds, B, k, tau_max) alone.
"""
from __future__ import annotations

import os
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import sampler as S


def _chunks(first, count, chunk):
    return [(first + o, min(chunk, count - o)) for o in range(0, count, chunk)]


def _gen(args):
    first, count, kw = args
    return S.halting_programs(count, first=first, **kw)


def program_source(L: int, seed: int, pid: int, ell: int = 10, s: int = 2) -> str:
    """The array-language source of program `pid` (its tokens, space separated)."""
    return " ".join(S.fun_tokens(S.sample_fun(L, seed, pid, ell, s)))


def busy_beaver_search(rounds: int, batch: int, k: int = 16, L: int = 100, seed: int = 6,
                       tau_max: int = 10 ** 5, w: int = 32, n: int = 250, ell: int = 10, s: int = 2,
                       read_inputs: bool = False, workers: int | None = None, chunk: int = 1 << 14,
                       stream=None) -> dict:
    """Run `rounds` rounds of `batch` programs; returns the best k halting
    programs found (tau_h, program id, source) and timing."""
    from . import rasp as R
    workers = workers or (os.cpu_count() or 1)
    kw = dict(L=L, seed=seed, w=w, n=n, ell=ell, s=s, cap=tau_max, read_inputs=read_inputs)
    t0 = time.perf_counter()
    gen_wait = gpu_s = 0.0
    best: list[tuple[int, int]] = []          # (-tau_h, program id)
    steps_total = 0
    halted_total = 0
    with ThreadPoolExecutor(workers) as ex:
        def submit(r):
            return [ex.submit(_gen, (f, c, kw)) for f, c in _chunks(r * batch, batch, chunk)]

        pending = submit(0)
        b = None
        for r in range(rounds):
            tw = time.perf_counter()
            wl = S.concat([f.result() for f in pending])
            gen_wait += time.perf_counter() - tw
            if r + 1 < rounds:
                pending = submit(r + 1)           # overlaps this round's device work
            if b is None:
                b = R.Batch(wl.mem_words, wl.ell, wl.s, word_bits=wl.w, stream=stream)
            tg = time.perf_counter()
            b.load_workload(wl)
            b.run()
            tau, vm = b.top_halting(k)
            st = b.stats()
            gpu_s += time.perf_counter() - tg
            steps_total += st["vm_steps"]
            halted_total += st["halted"]
            best += [(-int(t), r * batch + int(v)) for t, v in zip(tau, vm)]
            best = sorted(best)[:k]
        if b is not None:
            b.close()
    wall = time.perf_counter() - t0
    return dict(best=[(-nt, pid, program_source(L, seed, pid, ell, s)) for nt, pid in best],
                programs=rounds * batch, halted=halted_total, vm_steps=steps_total, wall_s=wall,
                gpu_s=gpu_s, gen_wait_s=gen_wait, programs_per_s=rounds * batch / wall)
