"""Bounded device waits run out without a fault (needs a GPU).

The SMEM-staged kernel waits for each bulk copy of a VM's memory with a
poll limit that is a kernel argument. RASP_FAULT_INJECT=wait (read by the
host at launch) sets that limit to 0 polls, so the wait gives up at once: the
kernel flags the expiry, lets the copies it issued land, and returns; the
host sees RASP_EDEVICE and the CUDA context stays usable."""
import numpy as np
import pytest

from paper_2604_12902_gb300 import workloads as W
from tests.helpers import assert_same_state, oracle_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rasp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12902_gb300 import rasp as R
    R.lib()
    return R


def test_staged_wait_limit_runs_out_and_is_reported(rasp, monkeypatch):
    R = rasp
    wl = W.random_programs(num_vms=512, seed=21)
    monkeypatch.setenv("RASP_FAULT_INJECT", "wait")
    with R.Batch(wl.mem_words, wl.ell, wl.s, flags=R.SCHED_PERSIST) as b:
        b.load_workload(wl)
        b.run()
        with pytest.raises(R.RaspError) as e:
            b.sync()
        assert e.value.code == R.RASP_EDEVICE
        assert "bounded wait expired" in str(e.value)
    monkeypatch.delenv("RASP_FAULT_INJECT")
    # the context is usable: the same batch on a fresh batch object runs to the oracle's state
    st, _ = oracle_state(wl)
    with R.Batch(wl.mem_words, wl.ell, wl.s, flags=R.SCHED_PERSIST) as b:
        b.load_workload(wl)
        b.run()
        assert_same_state(b.read_state(), st, wl.ell, wl.s, what="after an expired wait")
