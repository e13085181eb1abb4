"""rasp_run_static: the entry point for callers that cannot allocate.

Callers that record CUDA graphs, that live inside another framework's
memory manager, or that run real-time loops cannot call cudaMalloc when they
advance machines. rasp_run_static takes their own device buffers and a
fixed scratch area inside the library, and allocates nothing. These tests
check, through the C ABI, that two calls in a row on such a caller-owned
state store give bit-for-bit the state that rasp_run gives on the same
machines, and that sizes beyond the scratch capacity are refused.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U64 = (1 << 64) - 1


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12902_gb300 import rasp as R
    R.lib()
    return torch, R


def _caller_store(torch, wl, c0):
    """The caller's own device buffers, in the layout rasp_run_static documents."""
    V = wl.num_vms
    n = wl.mem_words.astype(np.int64)
    npad = (n + 1) & ~1
    mem_off = np.zeros(V, np.int64)
    mem_off[1:] = np.cumsum(npad[:-1])
    mem = np.zeros(int(npad.sum()), np.int64)
    src = np.concatenate([[0], np.cumsum(n)])
    for v in range(V):
        mem[mem_off[v]:mem_off[v] + n[v]] = c0["mem"][src[v]:src[v + 1]]
    lp, sp = (wl.ell + 1) & ~1, (wl.s + 1) & ~1
    tape = np.zeros((V, lp), np.int64)
    for v in range(V):
        x = wl.tape_of(v)
        tape[v, :len(x)] = x
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return dict(i=dev(c0["i"]), a=dev(c0["a"]), steps=dev(c0["steps"].view(np.int64)),
                cap=dev(wl.caps.view(np.int64)), status=dev(c0["status"]), uhead=dev(c0["uhead"].view(np.int32)),
                ylen=dev(c0["ylen"].view(np.int32)), n=dev(wl.mem_words.view(np.int32)), mem_off=dev(mem_off),
                mem=dev(mem), tape=dev(tape.reshape(-1)), y=dev(np.zeros(V * sp, np.int64)),
                mem_off_h=mem_off, sp=sp)


def _run_static(torch, R, st, wl, budget, err):
    run = R.rasp_static_run(*(ctypes.c_void_p(st[k].data_ptr()) for k in
                              ("i", "a", "steps", "cap", "status", "uhead", "ylen", "n", "mem_off", "mem",
                               "tape", "y")),
                            wl.num_vms, 64, 0, wl.ell, wl.s, budget,
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                            ctypes.cast(err, ctypes.c_char_p), len(err), 0)
    return R.rasp_run_static(run)


def _assert_same(torch, st, ref, wl, what):
    torch.cuda.synchronize()
    h = {k: st[k].cpu().numpy() for k in ("i", "a", "steps", "status", "uhead", "ylen", "mem", "y")}
    assert np.array_equal(h["i"], ref["i"]), what
    assert np.array_equal(h["a"], ref["a"]), what
    assert np.array_equal(h["steps"].view(np.uint64), ref["steps"]), what
    assert np.array_equal(h["status"], ref["status"]), what
    assert np.array_equal(h["uhead"].view(np.uint32), ref["uhead"]), what
    assert np.array_equal(h["ylen"].view(np.uint32), ref["ylen"]), what
    assert np.array_equal(h["y"].reshape(wl.num_vms, st["sp"])[:, :wl.s], ref["y"]), what
    n = wl.mem_words.astype(np.int64)
    idx = np.concatenate([np.arange(o, o + k) for o, k in zip(st["mem_off_h"], n)])
    assert np.array_equal(h["mem"][idx], ref["mem"]), what


def test_static_run_matches_rasp_run_on_two_calls(env):
    torch, R = env
    from paper_2604_12902_gb300 import workloads as W
    wl = W.template_programs(num_vms=20000, seed=3)
    with R.Batch(wl.mem_words, wl.ell, wl.s) as b:
        b.load_workload(wl)
        c0 = b.read_state()
        b.run(150)
        ref1 = b.read_state()
        b.run()
        ref2 = b.read_state()
    st = _caller_store(torch, wl, c0)
    err = ctypes.create_string_buffer(256)
    assert _run_static(torch, R, st, wl, 150, err) == R.RASP_OK, err.value
    _assert_same(torch, st, ref1, wl, "first call (budget 150)")
    assert _run_static(torch, R, st, wl, U64, err) == R.RASP_OK, err.value
    _assert_same(torch, st, ref2, wl, "second call (to completion)")
    assert int((ref2["status"] == R.HALTED).sum()) == wl.num_vms


def test_static_run_refuses_more_vms_than_its_scratch(env):
    torch, R = env
    run = R.rasp_static_run()
    run.num_vms = R.RASP_STATIC_MAX_VMS + 1
    run.word_bits = 64
    err = ctypes.create_string_buffer(256)
    run.err_buf = ctypes.cast(err, ctypes.c_char_p)
    run.err_buf_size = len(err)
    assert R.rasp_run_static(run) == R.RASP_EINVAL
    assert b"exceeds the static scratch capacity" in err.value
