"""The generate -> run -> filter loop (search.busy_beaver_search) on the CPU:
the device batch is replaced by a stand-in that runs the oracle and selects
the top k with numpy, so what is checked is the loop's own logic -- program
ids across rounds, the merge of the per-round top k (ties to the smaller
id), the totals, and that the reported source is the program that ran."""
import os

import numpy as np

from paper_2604_12902_gb300 import dsl, sampler as S


def _top(steps, status, k):
    ids = np.nonzero(status == 1)[0]
    order = np.lexsort((ids, -steps[ids].astype(np.int64)))
    sel = ids[order[:k]]
    return steps[sel], sel.astype(np.uint32)


class OracleBatch:
    """The subset of rasp.Batch the search loop uses, computed by the oracle."""

    def __init__(self, mem_words, ell, s, word_bits=64, stream=None):
        self.w = word_bits
        self.st = None

    def load_workload(self, wl):
        self.wl = wl

    def run(self):
        from tests.helpers import oracle_state
        self.st, _ = oracle_state(self.wl, threads=os.cpu_count() or 1)

    def top_halting(self, k):
        return _top(self.st.steps, self.st.status, k)

    def stats(self):
        return {"vm_steps": int(self.st.steps.sum()), "halted": int((self.st.status == 1).sum())}

    def close(self):
        pass


def test_search_loop_logic_with_an_oracle_batch(monkeypatch):
    from paper_2604_12902_gb300 import rasp, search
    from tests.helpers import oracle_state
    monkeypatch.setattr(rasp, "Batch", OracleBatch)
    rounds, batch, k, L, cap = 4, 1500, 10, 60, 5000
    res = search.busy_beaver_search(rounds, batch, k=k, L=L, seed=12, tau_max=cap, workers=3, chunk=400)
    whole = S.halting_programs(rounds * batch, L=L, seed=12, cap=cap)
    st, _ = oracle_state(whole, threads=os.cpu_count() or 1)
    want_t, want_v = _top(st.steps, st.status, k)
    assert [t for t, _, _ in res["best"]] == [int(t) for t in want_t]
    assert [p for _, p, _ in res["best"]] == [int(v) for v in want_v]
    assert res["programs"] == rounds * batch
    assert res["vm_steps"] == int(st.steps.sum()) and res["halted"] == int((st.status == 1).sum())
    assert len({p for _, p, _ in res["best"]}) == k
    for t, pid, src in res["best"]:
        low = dsl.lower(dsl.parse(src), ell=10, s=2, mu=10)
        words = np.array([((x + (1 << 63)) % (1 << 64)) - (1 << 63) for x in low.words], np.int64)
        assert np.array_equal(words, whole.program_of(pid))

