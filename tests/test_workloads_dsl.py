"""Input generators and the array-language lowering (host logic, no GPU)."""
import numpy as np
import pytest

from oracle import oracle
from paper_2604_12902_gb300 import dsl, workloads as W
from tests.helpers import ADD, BNZ, LOD, MUL, PRI, RD, STO, busy_beavers


def test_philox_known_answers():
    """Known-answer vectors of Philox4x32-10 (Salmon et al. 2011, Random123 kat_vectors)."""
    f = 0xFFFFFFFF
    cases = [((0, 0, 0, 0, 0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
             ((f, f, f, f, f, f), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
             ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344, 0xA4093822, 0x299F31D0),
              (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1))]
    for args, want in cases:
        assert tuple(int(x) for x in W.philox4x32(*args)) == want


def test_draws_depend_only_on_vm_and_index():
    ids = np.array([5, 0, 1 << 33, 7], np.uint64)
    full = W.draws(9, 3, ids, 11)
    assert np.array_equal(full[:, :5], W.draws(9, 3, ids, 5))
    assert np.array_equal(full[2], W.draws(9, 3, ids[2:3], 11)[0])
    assert not np.array_equal(full, W.draws(10, 3, ids, 11))
    assert not np.array_equal(full, W.draws(9, 4, ids, 11))


def test_uniform_int_range():
    u = W.draws(1, 1, np.arange(1000, dtype=np.uint64), 64)
    x = W.uniform_int(u, -100, 100)
    assert x.min() == -100 and x.max() == 100
    y = W.log_uniform_int(u, 16, 4096)
    assert y.min() >= 16 and y.max() <= 4096


def test_random_programs_shape():
    wl = W.random_programs(num_vms=1024)
    assert wl.programs.shape == (1024 * 64,)
    ops = wl.programs[0::2]
    assert ops.min() == 1 and ops.max() == 7
    assert wl.programs[1::2].min() == 0 and wl.programs[1::2].max() == 63
    assert wl.tapes.min() >= -100 and wl.tapes.max() <= 100
    sub = W.random_programs(num_vms=10, first_vm=100)
    assert np.array_equal(sub.programs, wl.programs[100 * 64:110 * 64])


def test_template_chunking_and_subset():
    a = W.template_programs(num_vms=300, chunk=64)
    b = W.template_programs(num_vms=300, chunk=1000)
    assert np.array_equal(a.programs, b.programs) and np.array_equal(a.tapes, b.tapes)
    c = W.template_programs(num_vms=50, first_vm=250)
    assert np.array_equal(c.programs, a.programs[250 * 128:])


def test_template_programs_halt_and_take_expected_steps():
    """Every template program halts within the cap, after
    T + sum f + sum_k (7 + T_k (8 + b_k)) + 2 steps; the structure is read
    back from the words (LOD T; STO c opens loop k)."""
    wl = W.template_programs(num_vms=2000)
    st, _ = oracle.run_packed(wl.programs, wl.prog_off, wl.mem_words, wl.tapes, wl.tape_off,
                              wl.ell, wl.s, caps=wl.caps, threads=4)
    assert np.all(st.status == oracle.HALTED)
    I = 64
    for v in range(0, 2000, 97):
        p = wl.program_of(v).reshape(I, 2)
        assert list(p[:16, 0]) == [RD] * 16 and list(p[:16, 1]) == list(range(128, 144))
        assert list(p[-3:, 0]) == [PRI, PRI, 0]
        steps, k = 16 + 2, 16
        while k < I - 3:
            if p[k, 0] == LOD and p[k + 1, 0] == STO and 144 <= p[k + 1, 1] < 147 and p[k + 4, 0] == BNZ:
                T = int(p[k, 1])
                b = (int(p[k + 6, 1]) // 2) - k - 12
                steps += 7 + T * (8 + b)
                k += 12 + b
            else:
                steps += 1
                k += 1
        assert int(st.steps[v]) == steps


def test_lowering_matches_rules():
    """Sec. 2.2: Get = LOD 0; ADD; G + Z = J STO nu LOD z ADD nu; Put appends STO;
    Fun appends PRI q_0 and HLT."""
    low = dsl.lower("fun f0(ipt: W ^ 1) -> W ^ 1 { opt[0] = ipt[0] + 3 }", ell=10, s=2, mu=10)
    nu, ipt, opt = 16, 21, 31
    assert low.m == 8 and low.layout == {"nu": nu, "ipt": ipt, "opt": opt, "scr": 33}
    assert low.words == [LOD, 0, ADD, ipt, STO, nu, LOD, 3, ADD, nu, STO, opt, PRI, opt, 0, 0]
    assert low.min_mem == 16 + 5 + 10 + 2 + 10


def test_lowering_control_flow():
    src = "fun f0(ipt: W ^ 2) -> W ^ 1 { whl ipt[1] { ife scr[0] { hlt } { scr[9] = 2 } } }"
    low = dsl.lower(src, ell=2, s=1, mu=10)
    w = low.words
    ops = w[0::2]
    # lh: LOD 0 ADD ipt1 BNZ lb LOD 1 BNZ le | lb: LOD 0 ADD scr0 BNZ lt (else) LOD 2 STO scr9
    #     LOD 1 BNZ le2 | lt: PRI q0 HLT | le2: LOD 1 BNZ lh | le: PRI q0 HLT
    assert ops == [LOD, ADD, BNZ, LOD, BNZ, LOD, ADD, BNZ, LOD, STO, LOD, BNZ, PRI, 0,
                   LOD, BNZ, PRI, 0]
    assert w[2 * 2 + 1] == 10 and w[2 * 4 + 1] == 32 and w[2 * 15 + 1] == 0
    assert w[2 * 7 + 1] == 24 and w[2 * 11 + 1] == 28
    assert low.address("scr", 19) == low.layout["scr"] + 9


def test_lowering_read_inputs_prepends_rd():
    name, tau, src = busy_beavers()[2]
    low = dsl.lower(src, ell=10, s=2, read_inputs=True)
    assert low.words[:6] == [RD, low.layout["ipt"], RD, low.layout["ipt"] + 1, RD, low.layout["ipt"] + 2]


def test_parser_rejects_bad_programs():
    for bad in ["fun f0(ipt: W ^ 0) -> W ^ 1 { hlt }",
                "fun f0(ipt: W ^ 1) -> W ^ 1 { ipt[0] = 1 }",
                "fun f0(ipt: W ^ 1) -> W ^ 1 { opt[0] = 1 ; }",
                "fun f0(ipt: W ^ 1) -> W ^ 1 { opt[10] = 1 }"]:
        with pytest.raises(SyntaxError):
            dsl.parse(bad)


def test_quick_start_example_results():
    """The Python quick-start example program (RD 14; LOD 5; ADD 14; STO 15;
    PRI 15; LOD 1; BNZ 12, n = 16, l = s = 2) halts after 6 steps with first
    output x + 5, on the example's inputs (7 -> 12, -3 -> 2), by the oracle."""
    from oracle import spec
    prog = [6, 14, 1, 5, 2, 14, 4, 15, 7, 15, 1, 1, 5, 12]
    for x, y1 in (([7], 12), ([-3], 2)):
        c = spec.initial(prog, [v % (1 << 64) for v in x], 16, 2, 2, 64)
        (i, a, M, u, y), steps, status = spec.run(c, 2, 2, 64, 10 ** 6)
        assert (status, steps, y[0], y[1]) == (1, 6, 1, y1)
