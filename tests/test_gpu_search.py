"""Generate -> run -> filter on the GPU: the device top-k of halting times
equals a numpy selection over the oracle's final states, and the search
loop's best programs equal those of running every drawn program through the
oracle. Needs a GPU."""
import os

import numpy as np
import pytest

from paper_2604_12902_gb300 import dsl, sampler as S, workloads as W
from tests.helpers import oracle_state

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def rasp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12902_gb300 import rasp as R
    R.lib()
    return R


def top_numpy(steps, status, k, ids=None):
    """The k halted entries with the largest steps, ties by smaller id."""
    ids = np.arange(len(steps)) if ids is None else np.asarray(ids)
    h = np.nonzero(status == 1)[0]
    order = np.lexsort((ids[h], -steps[h].astype(np.int64)))
    pick = h[order[:k]]
    return steps[pick].astype(np.uint64), ids[pick]


def test_top_halting_matches_numpy(rasp):
    wl = W.random_programs(num_vms=300_000, seed=41)     # > 256 blocks x 1024: several tiles per block
    st, _ = oracle_state(wl, threads=THREADS)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s) as b:
        b.load_workload(wl)
        b.run()
        for k in (1, 7, 64, 1024):
            tau, vm = b.top_halting(k)
            want_t, want_v = top_numpy(st.steps, st.status, k)
            assert np.array_equal(tau, want_t) and np.array_equal(vm, want_v), k
        with pytest.raises(rasp.RaspError):
            b.top_halting(0)
        with pytest.raises(rasp.RaspError):
            b.top_halting(1025)


def test_top_halting_with_few_halted(rasp):
    wl = W.random_programs(num_vms=40, seed=3)
    st, _ = oracle_state(wl)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s) as b:
        b.load_workload(wl)
        b.run()
        tau, vm = b.top_halting(64)
    assert len(tau) == int((st.status == 1).sum())
    want_t, want_v = top_numpy(st.steps, st.status, 64)
    assert np.array_equal(tau, want_t) and np.array_equal(vm, want_v)


def test_search_loop_equals_the_oracle(rasp):
    from paper_2604_12902_gb300 import search
    rounds, batch, k, L, cap = 3, 2500, 8, 60, 20_000
    res = search.busy_beaver_search(rounds, batch, k=k, L=L, seed=9, tau_max=cap, workers=4, chunk=1000)
    whole = S.halting_programs(rounds * batch, L=L, seed=9, cap=cap)
    st, _ = oracle_state(whole, threads=THREADS)
    want_t, want_v = top_numpy(st.steps, st.status, k)
    assert [t for t, _, _ in res["best"]] == [int(t) for t in want_t]
    assert [p for _, p, _ in res["best"]] == [int(v) for v in want_v]
    assert res["vm_steps"] == int(st.steps.sum()) and res["halted"] == int((st.status == 1).sum())
    for t, pid, src in res["best"]:
        low = dsl.lower(dsl.parse(src), ell=10, s=2, mu=10)       # the reported source is the program run
        words = np.array([((x + (1 << 63)) % (1 << 64)) - (1 << 63) for x in low.words], np.int64)
        assert np.array_equal(words, whole.program_of(pid))
