"""The halting experiment of Sec. 3 on the GPU: programs drawn uniformly by
token length, lowered by the Sec. 2.2 rules, run at w = 32 with n = 250,
l = 10, s = 2; every VM's final state equals the oracle's, and the device
histogram of tau_h equals a histogram of the oracle's states (bit-exact
counts). Needs a GPU."""
import os

import numpy as np
import pytest

from paper_2604_12902_gb300 import sampler as S
from tests.helpers import assert_same_state, oracle_state

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1
EDGES = np.concatenate([np.arange(0, 101), [1000, 10 ** 4, 10 ** 5, 10 ** 6, 1 << 62]]).astype(np.uint64)


@pytest.fixture(scope="module")
def rasp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12902_gb300 import rasp as R
    R.lib()
    return R


def expected_histogram(steps, status, edges):
    """Counts of halted VMs per [edges[k], edges[k+1]) and the other classes,
    written out with numpy from final states."""
    h = steps[status == 1]
    inside = (h >= edges[0]) & (h < edges[-1])
    idx = np.searchsorted(edges, h[inside], side="right") - 1
    counts = np.bincount(idx, minlength=len(edges) - 1).astype(np.uint64)
    other = np.array([(status == 0).sum(), (status == 2).sum(), (status >= 3).sum(), (~inside).sum()], np.uint64)
    return counts, other


@pytest.mark.parametrize("read_inputs", [False, True])
def test_halting_programs_match_the_oracle(rasp, read_inputs):
    wl = S.halting_programs(4096, L=100, seed=6, cap=100_000, read_inputs=read_inputs)
    st, _ = oracle_state(wl, threads=THREADS)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, word_bits=wl.w) as b:
        b.load_workload(wl)
        b.run()
        got = b.read_state()
        counts, other = b.halting_histogram(EDGES)
    assert_same_state(got, st, wl.ell, wl.s, what="halting w=32")
    want_c, want_o = expected_histogram(st.steps, st.status, EDGES)
    assert np.array_equal(counts, want_c)
    assert np.array_equal(other, want_o)
    assert 0 < want_o[1] < 4096 and int(want_c.sum()) > 0.5 * 4096


def test_halting_full_cap_histogram_and_sample(rasp):
    """2^17 programs to tau_max = 10^6: the device histogram equals numpy on
    the read-back state, and sampled VMs (timeouts included) equal the
    oracle."""
    wl = S.halting_programs_parallel(1 << 17, workers=THREADS, L=100, seed=7, cap=10 ** 6)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, word_bits=wl.w) as b:
        b.load_workload(wl)
        b.run()
        got = b.read_state(mem=False)
        counts, other = b.halting_histogram(EDGES)
    want_c, want_o = expected_histogram(got["steps"], got["status"], EDGES)
    assert np.array_equal(counts, want_c) and np.array_equal(other, want_o)
    rng = np.random.default_rng(1)
    ids = np.concatenate([rng.choice(wl.num_vms, 400, replace=False),
                          np.nonzero(got["status"] == 2)[0][:40]])
    sub = wl.subset(ids)
    st, _ = oracle_state(sub, threads=THREADS)
    part = {k: got[k][ids] for k in ("i", "a", "steps", "status", "uhead", "ylen", "y")}
    assert_same_state(part, st, wl.ell, wl.s, what="sampled halting VMs")


def test_histogram_rejects_bad_edges(rasp):
    wl = S.halting_programs(64, L=40, seed=1, cap=1000)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, word_bits=wl.w) as b:
        b.load_workload(wl)
        b.run()
        with pytest.raises(rasp.RaspError) as e:
            b.halting_histogram(np.array([0, 5, 5, 9], np.uint64))
        assert e.value.code == rasp.RASP_EINVAL
        with pytest.raises(rasp.RaspError):
            b.halting_histogram(np.array([3], np.uint64))
        counts, other = b.halting_histogram(np.array([0, 1 << 62], np.uint64))
        st = b.read_state(mem=False)
        assert int(counts[0]) == int((st["status"] == 1).sum())


def test_histogram_at_the_maximum_bin_count(rasp):
    """4096 unit bins (the documented maximum; the edges and counters need
    more than the default 48 KB of shared memory) equal numpy on the
    read-back state; 4097 bins are refused."""
    wl = S.halting_programs(20000, L=100, seed=8, cap=5000)
    edges = np.arange(0, 4097, dtype=np.uint64)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, word_bits=wl.w) as b:
        b.load_workload(wl)
        b.run()
        got = b.read_state(mem=False)
        counts, other = b.halting_histogram(edges)
        with pytest.raises(rasp.RaspError) as e:
            b.halting_histogram(np.arange(0, 4098, dtype=np.uint64))
        assert e.value.code == rasp.RASP_EINVAL
    want_c, want_o = expected_histogram(got["steps"], got["status"], edges)
    assert counts.shape == (4096,)
    assert np.array_equal(counts, want_c) and np.array_equal(other, want_o)
    assert int(want_c.sum()) > 10000 and int(np.count_nonzero(want_c)) > 30
