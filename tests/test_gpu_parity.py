"""CUDA path vs the CPU oracle, bit-exact, through the C ABI (needs a GPU)."""
import os

import numpy as np
import pytest

from paper_2604_12902_gb300 import dsl, workloads as W
from tests.helpers import (ADD, BNZ, LOD, MUL, PRI, RD, STO, U64, asm, assert_same_state,
                           batch, busy_beavers, checked_workload, oracle_state)

pytestmark = pytest.mark.gpu

SCHEDS = {"plain": 0x10, "persist": 0x20, "persist_gl": 0x30}
DISPATCH = {"select": 0x000, "vote": 0x100}
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def rasp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12902_gb300 import rasp as R
    R.lib()
    return R


def run_gpu(R, wl, flags=0, budget=U64, semantics=0, epoch=0, mem=True, steps_split=None):
    with R.Batch(wl.mem_words, wl.ell, wl.s, word_bits=wl.w, semantics=semantics,
                 flags=flags, epoch=epoch) as b:
        b.load_workload(wl)
        if steps_split:
            for t in steps_split:
                b.run(t)
        b.run(budget)
        got = b.read_state(mem=mem)
        stats = b.stats()
    return got, stats


def wl_from(programs, tapes, n, caps, ell, s, w=64, name="hand"):
    p, po, nn, t, to, cc = batch(programs, tapes, n, caps)
    return W.Workload(name, p, po, nn.astype(np.uint32), t, to,
                      cc if cc is not None else np.full(len(programs), U64, np.uint64), ell, s, w)


@pytest.mark.parametrize("sched", list(SCHEDS))
@pytest.mark.parametrize("disp", list(DISPATCH))
def test_random_programs_all_schedules(rasp, sched, disp):
    wl = W.random_programs(num_vms=1024, seed=1)
    st, _ = oracle_state(wl)
    got, stats = run_gpu(rasp, wl, SCHEDS[sched] | DISPATCH[disp])
    assert_same_state(got, st, wl.ell, wl.s, what="random/%s/%s" % (sched, disp))
    assert stats["vm_steps"] == int(st.steps.sum())


@pytest.mark.parametrize("sched", list(SCHEDS))
@pytest.mark.parametrize("disp", list(DISPATCH))
def test_template_programs_all_schedules(rasp, sched, disp):
    wl = W.template_programs(num_vms=20000, seed=2)
    st, _ = oracle_state(wl, threads=THREADS)
    got, _ = run_gpu(rasp, wl, SCHEDS[sched] | DISPATCH[disp])
    assert_same_state(got, st, wl.ell, wl.s, what="templates/%s/%s" % (sched, disp))


@pytest.mark.parametrize("epoch", [1, 7, 64])
def test_persistent_epoch_independence(rasp, epoch):
    wl = W.template_programs(num_vms=5000, seed=7)
    st, _ = oracle_state(wl)
    for sched in ("persist", "persist_gl"):
        got, _ = run_gpu(rasp, wl, SCHEDS[sched], epoch=epoch)
        assert_same_state(got, st, wl.ell, wl.s, what="epoch %d %s" % (epoch, sched))


def test_template_full_size_auto_schedule(rasp):
    """1,048,576 template programs, n = 256, cap 4096, the benchmark's launch
    configuration: every VM compared with the oracle."""
    wl = W.template_programs(num_vms=1 << 20, seed=2)
    st, h = oracle_state(wl, threads=THREADS, hist=True)
    got, stats = run_gpu(rasp, wl, 0)
    assert_same_state(got, st, wl.ell, wl.s, what="templates full")
    assert stats["halted"] == wl.num_vms


def test_random_full_size_stats(rasp):
    wl = W.random_programs(num_vms=1024, seed=1)
    st, h = oracle_state(wl, hist=True)
    for sched in SCHEDS.values():
        got, stats = run_gpu(rasp, wl, sched | 0x1000)
        assert stats["op_steps"][1:8] == [int(x) for x in h[1:8]]
        assert stats["pri_full"] == int(h[8]) and stats["bnz_taken"] == int(h[0])
        assert stats["halted"] == int((st.status == 1).sum())
        assert stats["timeout"] == int((st.status == 2).sum())


OPS = list(range(9))
ARGS = [0, 1, 2, 5, 1 << 63, U64]


@pytest.mark.parametrize("n,tape,w", [(6, [3, -2], 64), (8, [], 8), (6, [], 64), (8, [3, -2], 2)])
def test_exhaustive_tiny_programs(rasp, n, tape, w):
    instrs = [(o, a) for o in OPS for a in ARGS]
    progs = [[]] + [asm(x) for x in instrs] + [asm(x, y) for x in instrs for y in instrs]
    if n == 6 or w == 8:
        progs += [asm(x, y, z) for x in instrs for y in instrs for z in instrs]
    wl = wl_from(progs, [tape] * len(progs), n, 64, 2, 2, w=w, name="tiny")
    st, _ = oracle_state(wl, threads=THREADS)
    for sched in SCHEDS.values():
        got, _ = run_gpu(rasp, wl, sched)
        assert_same_state(got, st, 2, 2, what="tiny n=%d w=%d sched=%x" % (n, w, sched))


@pytest.mark.parametrize("w", [29, 32, 64])
def test_busy_beavers_on_gpu(rasp, w):
    bbs = busy_beavers()
    lows = [dsl.lower(src, ell=10, s=2) for _, _, src in bbs]
    wl = wl_from([l.words for l in lows], [[]] * 3, 256, 10 ** 6, 10, 2, w=w, name="bb")
    st, _ = oracle_state(wl)
    for sched in SCHEDS.values():
        got, _ = run_gpu(rasp, wl, sched)
        assert_same_state(got, st, 10, 2, what="bb w=%d" % w)
        if w == 29:
            assert [int(x) for x in got["steps"]] == [tau for _, tau, _ in bbs]


def test_checked_semantics_faults(rasp):
    wl = checked_workload()
    st, _ = oracle_state(wl, checked=True)
    counts = np.bincount(st.status, minlength=5)
    assert counts[3] > 50 and counts[4] > 500, counts          # both fault kinds occur
    for sched in SCHEDS.values():
        for disp in DISPATCH.values():
            got, stats = run_gpu(rasp, wl, sched | disp, semantics=1)
            assert_same_state(got, st, wl.ell, wl.s, what="checked %x" % (sched | disp))
            assert stats["fault_overflow"] == counts[3] and stats["fault_addr"] == counts[4]


def test_wrap_semantics_never_faults(rasp):
    wl = checked_workload()
    st, _ = oracle_state(wl)
    got, stats = run_gpu(rasp, wl, 0)
    assert_same_state(got, st, wl.ell, wl.s, what="wrap")
    assert stats["fault_overflow"] == 0 and stats["fault_addr"] == 0


@pytest.mark.parametrize("sched", list(SCHEDS))
def test_budget_and_resume(rasp, sched):
    wl = W.random_programs(num_vms=2048, seed=4, cap=300)
    for t1 in (0, 1, 13, 100):
        part, _ = oracle_state(wl, budget=t1)
        got, _ = run_gpu(rasp, wl, SCHEDS[sched], budget=t1)
        assert_same_state(got, part, wl.ell, wl.s, what="budget %d" % t1)
    full, _ = oracle_state(wl)
    got, _ = run_gpu(rasp, wl, SCHEDS[sched], steps_split=[5, 17, 17, 90])
    assert_same_state(got, full, wl.ell, wl.s, what="resumed")


@pytest.mark.parametrize("sched", list(SCHEDS))
def test_reset_repacks_c0_in_the_run(rasp, sched):
    """rasp_reset re-packs c_0 (Sec. 2.1) on the device from the loaded
    programs and tapes. 300,000 VMs is more than the resident lanes of the
    persistent schedules, so their queue and tail phases both run. Reading
    the state between reset and run shows c_0."""
    wl = W.random_programs(num_vms=300_000, seed=12)
    full, _ = oracle_state(wl, threads=THREADS)
    c0, _ = oracle_state(wl, budget=0, threads=THREADS)
    part, _ = oracle_state(wl, budget=37, threads=THREADS)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, flags=SCHEDS[sched]) as b:
        b.load_workload(wl)
        b.run()
        b.reset()
        got0 = b.read_state()
        assert (got0["status"] == 0).all(), "reset leaves every VM RUNNING"
        for key in ("i", "a", "steps", "uhead", "ylen"):
            assert not got0[key].any(), key
        assert np.array_equal(got0["mem"].view(np.uint64), c0.mem), "c_0 memory"
        assert not got0["y"].any()
        b.run()
        assert_same_state(b.read_state(), full, wl.ell, wl.s, what="reset+run %s" % sched)
        b.reset()
        b.run(37)
        assert_same_state(b.read_state(), part, wl.ell, wl.s, what="reset+run(37) %s" % sched)
        b.run()
        assert_same_state(b.read_state(), full, wl.ell, wl.s, what="reset+run(37)+run %s" % sched)
        b.reset()
        b.run()
        st = b.stats()
    assert st["vm_steps"] == int(full.steps.sum())


@pytest.mark.parametrize("flags,w", [(0x30 | 0x10000, 64), (0x30 | 0x100, 64), (0x30, 13), (0x30 | 0x20000, 64)])
def test_reset_then_run_matches_the_oracle(rasp, flags, w):
    """rasp_reset re-packs c_0 after a partial run; a run from there matches
    the oracle in every field, twice in a row: with budget rounds, with warp
    opcode voting, at w = 13 and with the per-step block."""
    wl = W.uneven_programs(num_vms=20000, seed=31, n_hi=1024, cap_hi=20000)
    wl.w = w
    full, _ = oracle_state(wl, threads=THREADS)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, word_bits=w, flags=flags) as b:
        b.load_workload(wl)
        b.run(50)
        for k in range(2):
            b.reset()
            b.run()
            assert_same_state(b.read_state(), full, wl.ell, wl.s, what="reset+run %d flags %#x w %d" % (k, flags, w))


def test_reset_repacks_shared_programs(rasp):
    """c_0 packed in the run kernel from a program shared by many VMs."""
    wl = W.shared_programs(num_programs=600, vms_per_program=256)
    full, _ = oracle_state(wl, threads=THREADS)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s, flags=SCHEDS["persist_gl"]) as b:
        b.load_workload(wl)
        b.run(100)
        b.reset()
        b.run()
        got = b.read_state()
    assert_same_state(got, full, wl.ell, wl.s, what="shared reset+run")


@pytest.mark.parametrize("w", [64, 32])
def test_long_runs_across_budget_rounds(rasp, w):
    """Countdown loops of up to ~320,000 steps with mixed caps (some VMs time
    out): the persistent schedule runs them in budget rounds with the still-
    running VMs compacted between rounds; one run, and a run split at budgets
    that fall inside rounds, both equal the oracle."""
    rng = np.random.default_rng(21)
    V = 2048
    progs, tapes = [], []
    for v in range(V):
        T = int(rng.integers(1, 40_000))
        progs.append(asm((LOD, T), (STO, 40), (LOD, 0), (ADD, 40), (BNZ, 12), (0, 0),
                         (LOD, -1), (ADD, 40), (STO, 40), (LOD, 1), (BNZ, 4), (PRI, 40)))
        tapes.append([])
    caps = rng.integers(1_000, 400_000, size=V).astype(np.uint64)
    caps[::7] = U64                                   # some VMs uncapped
    wl = wl_from(progs, tapes, 64, caps, 0, 2, w=w, name="countdown")
    full, _ = oracle_state(wl, threads=THREADS)
    assert (full.status == 2).any() and (full.status == 1).any()
    for flags in (SCHEDS["persist_gl"] | 0x10000, 0x10000, SCHEDS["persist_gl"]):   # forced rounds, and one launch
        got, _ = run_gpu(rasp, wl, flags)
        assert_same_state(got, full, wl.ell, wl.s, what="rounds w=%d flags %#x" % (w, flags))
    got, _ = run_gpu(rasp, wl, 0x10000, steps_split=[3_000, 50_000, 200_001])
    assert_same_state(got, full, wl.ell, wl.s, what="rounds split w=%d" % w)


def test_checkpoint_restore_roundtrip(rasp):
    wl = W.template_programs(num_vms=3000, seed=9)
    full, _ = oracle_state(wl)
    with rasp.Batch(wl.mem_words, wl.ell, wl.s) as b:
        b.load_workload(wl)
        b.run(150)
        snap = b.read_state()
    with rasp.Batch(wl.mem_words, wl.ell, wl.s) as b2:
        b2.load_workload(wl)                 # tapes and caps; state is then overwritten
        b2.load_state(snap)
        b2.run()
        got = b2.read_state()
    assert_same_state(got, full, wl.ell, wl.s, what="restored")


def test_ragged_memory_sizes_and_odd_tapes(rasp):
    """Mixed n across every bucket (odd n, n = 1, n >= 2048), odd l and s,
    empty programs, cap 0."""
    rng = np.random.default_rng(3)
    ns = [1, 2, 3, 5, 7, 63, 64, 65, 127, 255, 256, 257, 511, 700, 1000, 1500, 3000, 4096]
    progs, tapes, nn, caps = [], [], [], []
    for v in range(1500):
        n = ns[v % len(ns)]
        m = int(rng.integers(0, n // 2 + 1))
        ops = rng.integers(0, 9, size=m)
        args = rng.integers(-2, n + 2, size=m)
        progs.append([int(x) for pair in zip(ops, args) for x in pair])
        tapes.append([int(x) for x in rng.integers(-50, 50, size=int(rng.integers(0, 4)))])
        nn.append(n)
        caps.append(int(rng.choice([0, 1, 50, 400])))
    wl = wl_from(progs, tapes, nn, caps, 3, 5)
    st, _ = oracle_state(wl)
    for sched in SCHEDS.values():
        for disp in DISPATCH.values():
            got, _ = run_gpu(rasp, wl, sched | disp)
            assert_same_state(got, st, 3, 5, what="ragged %x" % (sched | disp))


def test_instruction_counter_wraps_at_word_boundary(rasp):
    """Place i just below 2^w (via a restored state) so that i (+) 1 and i (+) 2 wrap."""
    from oracle import oracle
    for w, n in ((64, 250), (64, 256), (16, 250), (8, 7)):
        wl = wl_from([asm((LOD, 3))] * 4, [[]] * 4, n, 40, 1, 1, w=w)
        mask = (1 << w) - 1
        st = oracle.pack(wl.programs, wl.prog_off, wl.mem_words, wl.tapes, wl.tape_off, 1, 1, w=w)
        i0 = [mask, mask - 1, mask - 2, mask - 3]
        rng = np.random.default_rng(w + n)
        st.i[:] = np.array(i0, np.uint64)
        st.mem[:] = rng.integers(0, 8, size=st.mem.shape[0]).astype(np.uint64)
        with rasp.Batch(wl.mem_words, 1, 1, word_bits=w) as b:
            b.load_workload(wl)
            b.load_state(dict(i=st.i.view(np.int64), mem=st.mem.view(np.int64)))
            b.run()
            got = b.read_state()
        oracle.run(st, caps=wl.caps)
        assert_same_state(got, st, 1, 1, what="wrap w=%d n=%d" % (w, n))


def test_shared_programs_match_expanded(rasp):
    base = W.template_programs(num_vms=64, seed=5, instructions=48, mem_words=224, tape_len=8, loops_hi=2)
    V = 64 * 50
    prog_of_vm = np.repeat(np.arange(64, dtype=np.uint32), 50)
    ids = np.arange(V, dtype=np.uint64)
    tape = W.uniform_int(W.draws(5, 9, ids, 8), -50, 50).reshape(-1)
    wl = W.Workload("shared", base.programs, base.prog_off, np.full(V, 224, np.uint32), tape,
                    np.arange(V + 1, dtype=np.uint64) * 8, np.full(V, 2048, np.uint64), 8, 8,
                    prog_of_vm=prog_of_vm)
    st, _ = oracle_state(wl)
    for sched in SCHEDS.values():
        got, _ = run_gpu(rasp, wl, sched)
        assert_same_state(got, st, 8, 8, what="shared %x" % sched)


def slab_over_4gib_workload():
    """One VM whose M slab is larger than 4 GiB (n = 2^29 + 6 words), then a
    small VM whose slab starts past 4 GiB. The big VM keeps a counter, a
    data word and a self-written instruction at the top of its memory, reads
    them through operands j >= n (j mod n), jumps to the instruction it wrote
    at n - 2, whose i (+) 2 = n fetches M[0] again (circular fetch), and
    leaves through a jump to n - 1, where the pair <M[n-1], M[0]> is an
    invalid opcode (a fixed point)."""
    N = (1 << 29) + 6
    big = asm((LOD, 1), (ADD, N - 4), (STO, N - 4),        # 0: c <- c + 1
              (ADD, 41), (BNZ, 14),                        # 6: c - 3 != 0 -> body
              (LOD, 1), (BNZ, N - 1),                      # 10: exit through <M[n-1], M[0]>
              (RD, N - 5), (LOD, 0), (ADD, 2 * N - 3),     # 14: body
              (ADD, N - 5), (MUL, 3 * N - 5), (STO, N - 3), (PRI, 4 * N - 3),
              (LOD, MUL), (STO, N - 2), (LOD, N - 3), (STO, N - 1),   # 28: M[n-2..] <- MUL n-3
              (LOD, 1), (BNZ, N - 2),                      # 36: run it; i (+) 2 = n
              (LOD, -3))                                   # 40: M[41] = -3, never run
    small = asm((RD, 10), (LOD, 5), (ADD, 10), (STO, 11), (PRI, 11), (LOD, 1), (BNZ, 12))
    return wl_from([big, small], [[11, -7, 5], [9]], [N, 16], [10 ** 4, 100], 3, 3), N


def test_memory_slab_over_4gib(rasp):
    """Byte offsets past 2^32 inside one slab and between slabs, on every
    schedule (a forced staged schedule falls back to HBM slabs for this n)."""
    wl, N = slab_over_4gib_workload()
    st, _ = oracle_state(wl)
    assert list(st.status) == [1, 1] and st.steps[0] > 40        # both halt, the loop ran
    assert st.mem[N - 4] == 3 and st.mem[N - 2] == MUL
    for sched in SCHEDS.values():
        got, _ = run_gpu(rasp, wl, sched)
        assert_same_state(got, st, 3, 3, what="slab > 4 GiB %x" % sched)
        del got


def test_argument_errors(rasp):
    R = rasp
    wl = W.random_programs(num_vms=8)
    with pytest.raises(R.RaspError) as e:
        R.Batch(wl.mem_words, 4, 8, word_bits=1)
    assert e.value.code == R.RASP_EINVAL
    with pytest.raises(R.RaspError):
        R.Batch(wl.mem_words, 4, 8, word_bits=32, semantics=R.CHECKED)
    with pytest.raises(R.RaspError):
        R.Batch(np.array([64, 0], np.uint32), 4, 8)
    with R.Batch(wl.mem_words, 4, 8) as b:
        with pytest.raises(R.RaspError) as e:
            b.run()
        assert e.value.code == R.RASP_ESTATE
        bad = wl.prog_off.copy()
        bad[1] = 3
        with pytest.raises(R.RaspError):
            b.load_programs(wl.programs, bad)
        with pytest.raises(R.RaspError):                          # program longer than n
            b.load_programs(np.zeros(8 * 66, np.int64), np.arange(9, dtype=np.uint64) * 66)
        b.load_programs(wl.programs, wl.prog_off)
        with pytest.raises(R.RaspError):                          # |x| > l
            b.load_inputs(np.zeros(40, np.int64), np.arange(9, dtype=np.uint64) * 5)
        b.load_inputs(wl.tapes, wl.tape_off, wl.caps)
        b.run()
        with pytest.raises(R.RaspError):
            b.read_state(first=5, count=10)


def test_self_modifying_programs_across_kernel_switches(rasp):
    """Self-modifying programs switched between the HBM-slab epoch loop and
    the plain kernel midway (per-bucket plans pinned between runs), in both
    orders, then reset and run again: every VM equal to the oracle's."""
    R = rasp
    wl = W.random_programs(num_vms=2048, seed=21)
    st, _ = oracle_state(wl)
    cuts = (40, 90, 160)
    parts = [oracle_state(wl, budget=c)[0] for c in cuts]
    for order in ((0x30, 0x10, 0x30, 0x10), (0x10, 0x30, 0x10, 0x30)):
        with R.Batch(wl.mem_words, wl.ell, wl.s) as b:
            b.load_workload(wl)
            for rep in range(2):
                for j, (c, part) in enumerate(zip(cuts, parts)):
                    b.plan_bucket(b.describe()["buckets"][0]["index"], order[j])
                    b.run(c)
                    if j == 1:
                        assert_same_state(b.read_state(), part, wl.ell, wl.s, what="order %s, %d steps" % (order, c))
                b.plan_bucket(b.describe()["buckets"][0]["index"], order[3])
                b.run()
                assert_same_state(b.read_state(), st, wl.ell, wl.s, what="order %s, to the end" % (order,))
                b.reset()


@pytest.mark.parametrize("w", [32, 20, 5])
def test_narrow_words_checkpoint_and_schedules(rasp, w):
    """w <= 32: M is held in 4-byte words on the plain and HBM-slab
    schedules (8-byte words on the shared-program and SMEM-staged ones).
    Self-modifying programs on every schedule, a checkpoint read midway
    (M widened to int64), restored into a fresh batch and run on: every VM
    equal to the oracle's."""
    R = rasp
    wl = W.random_programs(num_vms=1500, seed=23)
    wl.w = w
    st, _ = oracle_state(wl)
    part, _ = oracle_state(wl, budget=50)
    for flags, bytes_ in ((0x00, 4), (0x10, 4), (0x30, 4), (0x20, 8), (0x30 | 0x100, 4), (0x30 | 0x20000, 4)):
        with R.Batch(wl.mem_words, wl.ell, wl.s, word_bits=w, flags=flags) as b:
            assert b.describe()["word_bytes"] == bytes_
            b.load_workload(wl)
            b.run(50)
            ck = b.read_state()
            assert_same_state(ck, part, wl.ell, wl.s, what="w %d flags %#x at 50 steps" % (w, flags))
            b.run()
            assert_same_state(b.read_state(), st, wl.ell, wl.s, what="w %d flags %#x" % (w, flags))
        with R.Batch(wl.mem_words, wl.ell, wl.s, word_bits=w, flags=flags) as b2:
            b2.load_workload(wl)
            b2.load_state(ck)
            b2.run()
            assert_same_state(b2.read_state(), st, wl.ell, wl.s, what="w %d flags %#x restored" % (w, flags))


def test_programs_loaded_as_int32_words(rasp):
    """Programs whose words fit in 32 bits, loaded as int32 words and
    sign-extended on the device, give the same machines as int64 words:
    templates (negative immediates), self-modifying random programs at
    w = 64 and w = 32 (4-byte machine words), shared programs; a reset
    re-packs from the widened programs; a failed load leaves no programs."""
    R = rasp
    # Templates and shared programs fill at most half of M: their 4-byte
    # words stay as such (the pack reads them, the 8-byte copy is made only
    # for the shared-program kernel or a read-back of a lazily packed batch).
    # Random programs fill all of M: widened before the pack. rasp_describe
    # reports which.
    SHARED, GRAPH = 0x40, 0x4000
    cases = [(W.template_programs(num_vms=3000, seed=31), 64, 0), (W.template_programs(num_vms=3000, seed=34), 64, GRAPH),
             (W.template_programs(num_vms=3000, seed=35), 32, 0),
             (W.random_programs(num_vms=2000, seed=32), 64, 0), (W.random_programs(num_vms=2000, seed=33), 32, 0),
             (W.shared_programs(num_programs=64, vms_per_program=16), 64, 0),
             (W.shared_programs(num_programs=64, vms_per_program=16), 64, SHARED),
             (W.shared_programs(num_programs=64, vms_per_program=16), 64, SHARED | GRAPH)]
    for wl, w, flags in cases:
        wl.w = w
        assert np.all(np.abs(wl.programs) < (1 << 31))
        st, _ = oracle_state(wl)
        with R.Batch(wl.mem_words, wl.ell, wl.s, word_bits=w, flags=flags) as b:
            R.rasp_load_programs_i32(b.h, wl.programs.astype(np.int32), wl.prog_off, wl.prog_of_vm)
            b.load_inputs(wl.tapes, wl.tape_off, wl.caps)
            kept = 2 * int(wl.prog_off[-1]) <= int(((wl.mem_words.astype(np.uint64) + 1) // 2 * 2).sum())
            assert b.describe()["program_word_bytes"] == (4 if kept else 8), wl.name
            if flags & SHARED:
                b.run(20)                 # lazily packed: the read-back fills in the program words
                mid = b.read_state()
                assert mid["steps"].max() == 20
            b.run()
            what = "int32 programs, %s w %d flags %#x" % (wl.name, w, flags)
            assert_same_state(b.read_state(), st, wl.ell, wl.s, what=what)
            b.reset()
            b.run()
            assert_same_state(b.read_state(), st, wl.ell, wl.s, what="after reset, " + what)
            if wl.prog_of_vm is not None:
                b.reset()
                rep = b.autotune(reps=1)  # the shared-program trial reads the 8-byte words
                assert "shared" in [t["schedule"] for t in rep["trials"]]
                b.run()
                assert_same_state(b.read_state(), st, wl.ell, wl.s, what="after autotune, " + what)
            bad = wl.prog_off.copy()
            bad[1] = 3
            with pytest.raises(R.RaspError):
                R.rasp_load_programs_i32(b.h, wl.programs.astype(np.int32), bad, wl.prog_of_vm)
            with pytest.raises(R.RaspError) as e:
                b.run()
            assert e.value.code == R.RASP_ESTATE


@pytest.mark.parametrize("flags", [0x00, 0x4000], ids=["eager", "cuda-graph"])
def test_inputs_reloaded_midway_reset_the_read_head(rasp, flags):
    """rasp_load_inputs resets u_0 = 0 (applied by the next pack, or before
    u_0 is next read or run): reloading the tapes midway reads back u_0 = 0,
    and running on equals restoring the midway state with u_0 = 0."""
    R = rasp
    wl = W.template_programs(num_vms=2500, seed=41)
    with R.Batch(wl.mem_words, wl.ell, wl.s, flags=flags) as a, R.Batch(wl.mem_words, wl.ell, wl.s, flags=flags) as b:
        a.load_workload(wl)
        b.load_workload(wl)
        a.run(30)
        b.run(30)
        mid = b.read_state()
        assert mid["uhead"].max() > 0
        a.load_inputs(wl.tapes, wl.tape_off, wl.caps)
        after = a.read_state()
        assert after["uhead"].max() == 0
        for k in ("i", "a", "steps", "status", "mem"):
            assert np.array_equal(after[k], mid[k]), k
        a.load_inputs(wl.tapes, wl.tape_off, wl.caps)       # again, then straight into a run
        a.run()
        mid["uhead"][:] = 0
        b.load_state(mid)
        b.run()
        ga, gb = a.read_state(), b.read_state()
    for k in ga:
        assert np.array_equal(ga[k], gb[k]), k
