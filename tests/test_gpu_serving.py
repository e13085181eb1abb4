"""Serving: continuous batching of rollout requests in one device arena
(needs a GPU). A request's result must not depend on what else is running."""
import os

import numpy as np
import pytest

from paper_2604_12902_gb300 import workloads as W
from tests.helpers import assert_same_state, oracle_state

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def serving():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12902_gb300 import rasp as R, serving as S
    R.lib()
    return R, S


def request(size, k, seed=5):
    """A rollout request shaped like the uneven batch (sizes as in config 3)."""
    return W.uneven_programs(num_vms=size, seed=seed, first_vm=k * 200_000)


def wait(pool, t):
    import time
    for _ in range(200000):
        if pool.poll(t) == 2:
            return
        time.sleep(1e-4)
    raise AssertionError("request did not finish")


def test_request_same_alone_and_in_the_mix(serving):
    R, S = serving
    reqs = [request(n, k) for k, n in enumerate([3000, 20000, 1000, 7000, 12000])]
    A = reqs[0]
    with S.Pool(8 << 30, A.ell, A.s) as pool:
        t = pool.submit(A)
        wait(pool, t)
        alone = pool.read(t, mem=True)
        tickets = [pool.submit(r) for r in reqs[1:3]] + [pool.submit(A)] + [pool.submit(r) for r in reqs[3:]]
        res = {}
        for tk in tickets:
            wait(pool, tk)
        for tk, r in zip(tickets, reqs[1:3] + [A] + reqs[3:]):
            res[tk] = (r, pool.read(tk, mem=True))
    mixed = res[tickets[2]][1]
    for key in alone:
        assert np.array_equal(alone[key], mixed[key]), key
    st, _ = oracle_state(A, threads=THREADS)
    assert_same_state(alone, st, A.ell, A.s, what="request alone")
    r4, got4 = res[tickets[-1]]
    st4, _ = oracle_state(r4, threads=THREADS)
    assert_same_state(got4, st4, r4.ell, r4.s, what="request in the mix")


def test_admission_waits_for_memory(serving):
    R, S = serving
    reqs = [request(20000, k, seed=6) for k in range(5)]
    one = max(R.rasp_batch_bytes(R.rasp_config(64, 0, 16, 8, 0, 0, 0, 0, 0, 0, None, None, 0), r.mem_words)
              for r in reqs)
    with S.Pool(int(one * 2.2), reqs[0].ell, reqs[0].s) as pool:
        tickets = [pool.submit(r) for r in reqs]
        info = pool.info()
        assert info["waiting"] >= 2 and info["running"] <= 2
        outs = {}
        pending = list(tickets)
        while pending:
            for tk in list(pending):
                if pool.poll(tk) == 2:
                    outs[tk] = pool.read(tk)
                    pending.remove(tk)
        assert pool.info()["in_use"] == 0
    for tk, r in zip(tickets, reqs):
        st, _ = oracle_state(r, threads=THREADS)
        got = outs[tk]
        got["mem"] = None
        assert np.array_equal(got["steps"], st.steps) and np.array_equal(got["status"], st.status)


def test_poisson_short_run(serving):
    R, S = serving
    rng = np.random.default_rng(7)
    sizes = W.log_uniform_int(rng.integers(0, 1 << 32, size=12, dtype=np.uint64).astype(np.uint32), 1000, 20000)
    reqs = [request(int(n), k, seed=7) for k, n in enumerate(sizes)]
    with S.Pool(16 << 30, reqs[0].ell, reqs[0].s) as pool:
        out = S.poisson_run(pool, reqs, lam=200.0, duration=0.5, seed=1, keep_results=True)
    assert out["requests"] >= 40 and out["p50_ms"] > 0 and out["p99_ms"] >= out["p50_ms"]
    seen = {}
    for idx, res in out["results"]:
        if idx not in seen:
            seen[idx] = res
        else:
            for key in res:                                  # every replay of a request gives the same result
                assert np.array_equal(seen[idx][key], res[key]), key
    idx, res = out["results"][0]
    st, _ = oracle_state(reqs[idx], threads=THREADS)
    assert np.array_equal(res["steps"], st.steps) and np.array_equal(res["i"].view(np.uint64), st.i)


def test_cancel_a_waiting_request(serving):
    """A request still waiting for memory can be withdrawn; the others run to
    the same results as alone; an admitted request cannot be cancelled."""
    R, S = serving
    reqs = [request(20000, k, seed=8) for k in range(4)]
    one = max(R.rasp_batch_bytes(R.rasp_config(64, 0, 16, 8, 0, 0, 0, 0, 0, 0, None, None, 0), r.mem_words)
              for r in reqs)
    with S.Pool(int(one * 1.5), reqs[0].ell, reqs[0].s) as pool:
        tickets = [pool.submit(r) for r in reqs]
        assert pool.info()["waiting"] == 3
        pool.cancel(tickets[2])
        assert pool.info()["waiting"] == 2
        with pytest.raises(R.RaspError) as e:
            pool.cancel(tickets[0])                   # running
        assert e.value.code == R.RASP_ESTATE
        with pytest.raises(R.RaspError):
            pool.poll(tickets[2])                     # forgotten
        outs = {}
        for tk in (tickets[0], tickets[1], tickets[3]):
            wait(pool, tk)
            outs[tk] = pool.read(tk)
    for k in (0, 1, 3):
        st, _ = oracle_state(reqs[k], threads=THREADS)
        got = outs[tickets[k]]
        assert np.array_equal(got["steps"], st.steps) and np.array_equal(got["status"], st.status)


def test_next_done_hands_out_every_request_once(serving):
    R, S = serving
    reqs = [request(3000 + 500 * k, k, seed=10) for k in range(6)]
    with S.Pool(4 << 30, reqs[0].ell, reqs[0].s) as pool:
        tickets = [pool.submit(r) for r in reqs]
        assert pool.poll(tickets[0]) in (1, 2)          # a poll may see it finish first
        seen = []
        for _ in range(200000):
            t = pool.next_done()
            if t:
                seen.append(t)
                pool.read(t)
            if len(seen) == len(tickets):
                break
        assert sorted(seen) == sorted(tickets)
        assert pool.next_done() == 0


def test_submit_refuses_null_buffers(serving):
    """Requests whose buffers a waiting copy would misread are refused at
    submit (EINVAL), the pool stays usable."""
    import ctypes
    R, S = serving
    wl = request(500, 0)
    pool = S.Pool(1 << 28, wl.ell, wl.s)
    try:
        po = np.ascontiguousarray(wl.prog_off, np.uint64)
        to = np.ascontiguousarray(wl.tape_off, np.uint64)
        mem = np.ascontiguousarray(wl.mem_words, np.uint32)
        tape = np.ascontiguousarray(wl.tapes, np.int64)
        words = np.ascontiguousarray(wl.programs, np.int64)
        L = S._lib()
        t = ctypes.c_uint64(0)
        for w_ptr, t_ptr, nprog in ((None, R._p(tape), wl.num_vms), (R._p(words), None, wl.num_vms),
                                    (R._p(words), R._p(tape), 0)):
            q = S.rasp_request(w_ptr, R._p(po), nprog, None, t_ptr, R._p(to), None, R._p(mem), wl.num_vms,
                               R.U64_MAX)
            assert L.rasp_pool_submit(pool.h, ctypes.byref(q), ctypes.byref(t)) == R.RASP_EINVAL
        st, _ = oracle_state(wl, threads=THREADS)
        k = pool.submit(wl)
        wait(pool, k)
        assert_same_state(pool.read(k), st, wl.ell, wl.s, what="after refused submits")
    finally:
        pool.close()


def test_serving_kernel_returns_when_idle_and_relaunches(serving):
    """The serving kernel waits for new ring entries only a bounded time: once
    every request is read, every instance returns by itself; a request that
    arrives later is served by a new instance, with the oracle's result."""
    import time
    R, S = serving
    reqs = [request(2000 + 1000 * k, k, seed=12) for k in range(3)]
    with S.Pool(4 << 30, reqs[0].ell, reqs[0].s) as pool:
        for r in reqs[:2]:
            t = pool.submit(r)
            wait(pool, t)
            pool.read(t)
        t0 = time.time()
        while True:
            st = pool.stats()
            if st["kernel_returns"] == st["kernel_launches"]:
                break
            assert time.time() - t0 < 10, st
            time.sleep(0.01)
        assert st["admitted"] == 2 and st["completed"] == 2 and st["vms_in_flight"] == 0
        assert st["ring_published"] == reqs[0].num_vms + reqs[1].num_vms
        t = pool.submit(reqs[2])
        wait(pool, t)
        got = pool.read(t, mem=True)
        assert pool.stats()["kernel_launches"] == st["kernel_launches"] + 1
    ref, _ = oracle_state(reqs[2], threads=THREADS)
    assert_same_state(got, ref, reqs[2].ell, reqs[2].s, what="after the kernel returned")
