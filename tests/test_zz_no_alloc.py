"""rasp_run_static: the entry point for callers that cannot allocate.

Engines whose device memory belongs to another framework's allocator, and
real-time loops that must not allocate, cannot call cudaMalloc when they
advance machines. rasp_run_static takes their own device buffers and a fixed
scratch area inside the library, and allocates nothing. These tests check,
through the C ABI:
- two calls in a row on a caller-owned state store give bit for bit the state
  that rasp_run gives on the same machines;
- the same two calls match the CPU oracle at w = 64, 32 and 5 (WRAP) and
  under CHECKED semantics with both fault kinds;
- VMs whose n or mem_off break the layout rules are not run and are counted;
- sizes beyond the scratch capacity are refused.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from tests.helpers import U64, assert_same_state, checked_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12902_gb300 import rasp as R
    R.lib()
    return torch, R


def _c0(wl, checked=False):
    """c_0 of every VM from the oracle's pack (Sec. 2.1), words reduced to w bits."""
    from oracle import oracle
    progs, po = wl.expanded_programs()
    return oracle.pack(progs, po, wl.mem_words, wl.tapes, wl.tape_off, wl.ell, wl.s, w=wl.w, checked=checked)


def _caller_store(torch, wl, c0):
    """The caller's own device buffers, in the layout rasp_run_static documents:
    slabs padded to an even number of words, tapes and outputs of even stride."""
    V = wl.num_vms
    n = wl.mem_words.astype(np.int64)
    npad = (n + 1) & ~1
    mem_off = np.zeros(V, np.int64)
    mem_off[1:] = np.cumsum(npad[:-1])
    mem = np.zeros(int(npad.sum()), np.uint64)
    for v in range(V):
        mem[mem_off[v]:mem_off[v] + n[v]] = c0.memory(v)
    lp, sp = (wl.ell + 1) & ~1, (wl.s + 1) & ~1
    tape = np.zeros((V, lp), np.uint64)
    u = c0.u.reshape(V, wl.ell + 1)
    tape[:, :wl.ell] = u[:, 1:]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return dict(i=dev(c0.i.view(np.int64)), a=dev(c0.a.view(np.int64)), steps=dev(c0.steps.view(np.int64)),
                cap=dev(wl.caps.view(np.int64)), status=dev(c0.status), uhead=dev(u[:, 0].astype(np.int32)),
                ylen=dev(np.zeros(V, np.int32)), n=dev(wl.mem_words.view(np.int32)), mem_off=dev(mem_off),
                mem=dev(mem.view(np.int64)), tape=dev(tape.reshape(-1).view(np.int64)),
                y=dev(np.zeros(V * sp, np.int64)), rejected=dev(np.full(1, 7, np.int32)),
                mem_off_h=mem_off, sp=sp, mem_words=int(npad.sum()))


def _run_static(torch, R, st, wl, budget, err, semantics=0, num_vms=None, mem_words=None):
    run = R.rasp_static_run(*(ctypes.c_void_p(st[k].data_ptr()) for k in
                              ("i", "a", "steps", "cap", "status", "uhead", "ylen", "n", "mem_off", "mem",
                               "tape", "y")),
                            wl.num_vms if num_vms is None else num_vms, wl.w, semantics, wl.ell, wl.s, budget,
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                            ctypes.cast(err, ctypes.c_char_p), len(err), 0,
                            st["mem_words"] if mem_words is None else mem_words,
                            ctypes.c_void_p(st["rejected"].data_ptr()))
    return R.rasp_run_static(run)


def _read(torch, st, wl):
    """The caller's store as the library's read_state would give it."""
    torch.cuda.synchronize()
    h = {k: st[k].cpu().numpy() for k in ("i", "a", "steps", "status", "uhead", "ylen", "mem", "y", "rejected")}
    n = wl.mem_words.astype(np.int64)
    idx = np.concatenate([np.arange(o, o + k) for o, k in zip(st["mem_off_h"], n)])
    return {"i": h["i"], "a": h["a"], "steps": h["steps"].view(np.uint64), "status": h["status"],
            "uhead": h["uhead"].view(np.uint32), "ylen": h["ylen"].view(np.uint32),
            "y": h["y"].reshape(wl.num_vms, st["sp"])[:, :wl.s].reshape(-1), "mem": h["mem"][idx],
            "rejected": int(h["rejected"][0])}


def _assert_same(got, ref, what):
    for k in ("i", "a", "steps", "status", "uhead", "ylen", "y", "mem"):
        assert np.array_equal(np.asarray(got[k]).reshape(-1).view(np.uint8),
                              np.asarray(ref[k]).reshape(-1).view(np.uint8)), "%s: field %s" % (what, k)


def test_static_run_matches_rasp_run_on_two_calls(env):
    torch, R = env
    from paper_2604_12902_gb300 import workloads as W
    wl = W.template_programs(num_vms=20000, seed=3)
    with R.Batch(wl.mem_words, wl.ell, wl.s) as b:
        b.load_workload(wl)
        b.run(150)
        ref1 = b.read_state()
        b.run()
        ref2 = b.read_state()
    st = _caller_store(torch, wl, _c0(wl))
    err = ctypes.create_string_buffer(256)
    assert _run_static(torch, R, st, wl, 150, err) == R.RASP_OK, err.value
    got1 = _read(torch, st, wl)
    _assert_same(got1, ref1, "first call (budget 150)")
    assert got1["rejected"] == 0
    assert _run_static(torch, R, st, wl, U64, err) == R.RASP_OK, err.value
    _assert_same(_read(torch, st, wl), ref2, "second call (to completion)")
    assert int((ref2["status"] == R.HALTED).sum()) == wl.num_vms


def _cases():
    from paper_2604_12902_gb300 import workloads as W
    tmpl = W.template_programs(num_vms=8192, seed=3)
    r32 = W.random_programs(num_vms=4096, seed=5)
    r32.w = 32
    r5 = W.random_programs(num_vms=4096, seed=6)
    r5.w = 5
    return {"templates w64": (tmpl, 0), "random w32": (r32, 0), "random w5": (r5, 0),
            "checked w64": (checked_workload(4096, 12), 1)}


@pytest.mark.parametrize("case", ["templates w64", "random w32", "random w5", "checked w64"])
def test_static_run_matches_the_oracle_on_two_calls(env, case):
    """Masked (w < 64), CHECKED and the default instance of the static kernel,
    each on two calls in a row (a budget, then to completion), against the
    oracle in every field, statuses included."""
    torch, R = env
    from oracle import oracle
    wl, semantics = _cases()[case]
    checked = semantics == 1
    c0 = _c0(wl, checked=checked)
    first = c0.copy()
    oracle.run(first, caps=wl.caps, budget=100)
    final = first.copy()
    oracle.run(final, caps=wl.caps)
    if checked:
        counts = np.bincount(final.status, minlength=5)
        assert counts[3] > 20 and counts[4] > 200, counts        # both fault kinds occur
    st = _caller_store(torch, wl, c0)
    err = ctypes.create_string_buffer(256)
    for budget, want, what in ((100, first, "first call"), (U64, final, "second call")):
        assert _run_static(torch, R, st, wl, budget, err, semantics=semantics) == R.RASP_OK, err.value
        got = _read(torch, st, wl)
        assert got["rejected"] == 0
        assert_same_state(got, want, wl.ell, wl.s, what="%s, %s" % (case, what))


def test_static_run_skips_invalid_layouts(env):
    """A VM with n = 0, one with an odd mem_off and one whose slab ends past
    mem_words are not run (their state stays c_0) and are counted; the others
    run as the oracle says."""
    torch, R = env
    from oracle import oracle
    from paper_2604_12902_gb300 import workloads as W
    wl = W.template_programs(num_vms=256, seed=7)
    c0 = _c0(wl)
    want = c0.copy()
    oracle.run(want, caps=wl.caps)
    st = _caller_store(torch, wl, c0)
    bad = {3: "n", 5: "odd", 255: "past"}
    n = wl.mem_words.astype(np.int32).copy()
    n[3] = 0
    off = st["mem_off_h"].copy()
    off[5] += 1
    off[255] = st["mem_words"] - 2            # 256 words would end 254 words past mem
    st["n"] = torch.from_numpy(n).cuda()
    st["mem_off"] = torch.from_numpy(off).cuda()
    err = ctypes.create_string_buffer(256)
    assert _run_static(torch, R, st, wl, U64, err) == R.RASP_OK, err.value
    torch.cuda.synchronize()
    assert int(st["rejected"].cpu()[0]) == len(bad)
    status = st["status"].cpu().numpy()
    steps = st["steps"].cpu().numpy()
    for v in bad:
        assert status[v] == R.RUNNING and steps[v] == 0, v
    good = np.array([v for v in range(wl.num_vms) if v not in bad])
    assert np.array_equal(status[good], want.status[good])
    assert np.array_equal(steps[good].view(np.uint64), want.steps[good])
    a = st["a"].cpu().numpy().view(np.uint64)
    assert np.array_equal(a[good], want.a[good])


def test_static_run_refuses_bad_arguments(env):
    torch, R = env
    run = R.rasp_static_run()
    run.num_vms = R.RASP_STATIC_MAX_VMS + 1
    run.word_bits = 64
    err = ctypes.create_string_buffer(256)
    run.err_buf = ctypes.cast(err, ctypes.c_char_p)
    run.err_buf_size = len(err)
    assert R.rasp_run_static(run) == R.RASP_EINVAL
    assert b"exceeds the static scratch capacity" in err.value
    from paper_2604_12902_gb300 import workloads as W
    wl = W.template_programs(num_vms=64, seed=3)
    st = _caller_store(torch, wl, _c0(wl))
    assert _run_static(torch, R, st, wl, U64, err, mem_words=0) == R.RASP_EINVAL
    assert b"mem_words" in err.value
