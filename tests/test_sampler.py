"""The uniform program sampler of the halting experiment (Sec. 3) against
brute force: its string counts equal an explicit enumeration of the Sec. 2.2
grammar (every enumerated string accepted by the independent parser of
dsl.py), every sample has exactly L tokens and parses back to itself, and on
a small space the samples are uniform (chi-square)."""
import os

import numpy as np
import pytest

from paper_2604_12902_gb300 import dsl, sampler as S

REFG = [(a, "[", str(z), "]") for a in ("ipt", "scr", "opt") for z in range(10)]
REFP = [(a, "[", str(z), "]") for a in ("scr", "opt") for z in range(10)]
Z = [(str(z),) for z in range(10)]


def enumerate_grammar(maxlen):
    """All token strings of E, S, B by length, written out from the grammar."""
    E = {1: list(Z), 4: list(REFG)}
    E[6] = [g + (op,) + z for g in REFG for op in "+*" for z in Z]
    E[9] = [g + (op,) + h for g in REFG for op in "+*" for h in REFG]
    Sx, Bx = {}, {}
    for l in range(1, maxlen + 1):
        out = []
        for p in REFP:
            out += [p + ("=",) + e for e in E.get(l - 5, [])]
        for k in range(1, l - 9):
            for g in REFG:
                out += [("ife",) + g + ("{",) + b1 + ("}", "{") + b2 + ("}",)
                        for b1 in Bx.get(k, []) for b2 in Bx.get(l - 9 - k, [])]
        for g in REFG:
            out += [("whl",) + g + ("{",) + b + ("}",) for b in Bx.get(l - 7, [])]
        Sx[l] = out
        blk = list(out) + ([("hlt",)] if l == 1 else [])
        for k in range(1, l - 1):
            blk += [s + (";",) + b for s in Sx.get(k, []) for b in Bx.get(l - k - 1, [])]
        Bx[l] = blk
    return Sx, Bx


def test_counts_equal_explicit_enumeration_and_parse():
    maxlen = 15
    Sx, Bx = enumerate_grammar(maxlen)
    _, cS, cB = S._counts(maxlen)
    for l in range(1, maxlen + 1):
        assert len(set(Bx[l])) == len(Bx[l]) == cB[l], l
        assert len(Sx[l]) == cS[l], l
    for body in Bx[13][::97] + Bx[15][::211]:
        src = "fun f0 ( ipt : W ^ 2 ) -> W ^ 1 { " + " ".join(body) + " }"
        dsl.parse(src)                       # the independent parser accepts it
    assert S.count_programs(15 + 13, ell=10, s=2) == 9 * 2 * len(Bx[13])
    assert S.count_programs(15 + 13, ell=3, s=1) == 3 * 1 * len(Bx[13])


@pytest.mark.parametrize("L", [16, 40, 100])
def test_samples_have_L_tokens_and_parse_back(L):
    for k in range(60):
        f = S.sample_fun(L, seed=3, pid=k)
        toks = S.fun_tokens(f)
        assert len(toks) == L
        g = dsl.parse(" ".join(toks))
        assert (g.arity, g.out_arity, g.body) == (f.arity, f.out_arity, f.body)
        assert 1 <= f.arity <= 9 and 1 <= f.out_arity <= 2


def test_uniform_on_a_small_space():
    L = 21                                   # 9 x 2 x 200 = 3,600 programs
    n = S.count_programs(L)
    assert n == 3600
    draws = 36000
    seen = {}
    for k in range(draws):
        key = tuple(S.fun_tokens(S.sample_fun(L, seed=11, pid=k)))
        seen[key] = seen.get(key, 0) + 1
    assert len(seen) == n                    # every program reached
    exp = draws / n
    chi2 = sum((c - exp) ** 2 / exp for c in seen.values())
    dof = n - 1
    assert abs(chi2 - dof) < 5 * (2 * dof) ** 0.5, chi2


def test_deterministic_and_chunked_generation_equal():
    a = S.halting_programs(300, L=60, seed=5)
    b = S.concat([S.halting_programs(100, L=60, seed=5, first=o) for o in (0, 100, 200)])
    for f in ("programs", "prog_off", "tapes", "tape_off", "caps", "mem_words"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    lens = a.prog_off[1:] - a.prog_off[:-1]
    assert (lens % 2 == 0).all() and (lens // 2 * 2 + 5 + 10 + 2 + 10 <= 250).all()
    assert (a.tapes >= 0).all() and (a.tapes < 2 ** 32).all()


@pytest.mark.parametrize("L,read_inputs,w,n,first,e", [(100, False, 32, 250, 0, 0), (100, True, 64, 250, 9000, 0),
                                                       (60, False, 8, 250, 3, 0), (100, False, 32, 130, 0, 0),
                                                       (160, True, 32, 250, 11, 0), (100, False, 32, 250, 0, 1),
                                                       (100, True, 32, 130, 5, 2)])
def test_c_sampler_equals_the_python_definition(L, read_inputs, w, n, first, e):
    """progsampler.c draws the same programs and tapes as this module (word for
    word), including redraws when a lowering does not fit n words."""
    a = S.halting_programs(1500, L=L, read_inputs=read_inputs, w=w, n=n, first=first, impl="py", out_arity=e)
    b = S.halting_programs(1500, L=L, read_inputs=read_inputs, w=w, n=n, first=first, impl="c", out_arity=e)
    for f in ("programs", "prog_off", "tapes", "tape_off", "caps", "mem_words"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert a.meta["redraws"] == b.meta["redraws"]
    if n == 130:
        assert a.meta["redraws"] > 0


def test_minimum_halting_time_under_both_input_readings():
    """Sec. 3 / Fig. 1b report a minimum tau_h of 5 over the sampled programs.
    With the lowering pinned by App. B, the shortest run is an untaken
    ``ife`` on a zero word whose else-branch is ``hlt``: Get (2) + BNZ (1) +
    one PRI per output (e >= 1), so 3 + e = 4 when the program reads no
    input, and N + 3 + e = 5 (N >= 1 input words) when it first reads its
    inputs with RD. The sampler, lowering and oracle together must give
    exactly these minima."""
    from tests.helpers import oracle_state
    for read_inputs, want in ((False, 4), (True, 5)):
        wl = S.halting_programs(50000, L=100, seed=6, w=32, n=250, ell=10, s=2, cap=10 ** 4,
                                read_inputs=read_inputs)
        st, _ = oracle_state(wl, threads=os.cpu_count() or 1)
        halted = st.steps[st.status == 1]
        assert int(halted.min()) == want, (read_inputs, int(halted.min()))


def test_fixed_output_arity_keeps_the_body():
    """out_arity fixes e (every program ends in exactly e PRIs and the HLT
    pair) while the body drawn for program k stays the same."""
    from paper_2604_12902_gb300 import dsl
    for pid in range(200):
        drawn = S.sample_fun(100, 6, pid)
        fixed = S.sample_fun(100, 6, pid, out_arity=1)
        assert fixed.out_arity == 1 and fixed.body == drawn.body and fixed.arity == drawn.arity
    wl = S.halting_programs(300, out_arity=2, impl="c")
    for k in range(wl.num_vms):
        p = wl.programs[int(wl.prog_off[k]):int(wl.prog_off[k + 1])]
        assert list(p[-2:]) == [0, 0] and list(p[-6:-2:2]) == [dsl.PRI, dsl.PRI] and p[-8] != dsl.PRI
    with pytest.raises(ValueError):
        S.halting_programs(10, s=2, out_arity=3)


def _fig1b():
    """(counts for tau_h = 1..99, mass at >= 100, total) printed in Fig. 1b."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fig1b_counts.txt")
    c = np.zeros(100)
    long_ = 0
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        if k.isdigit():
            c[int(k)] = int(v)
        else:
            long_ += int(v)
    return c, long_, c.sum() + long_


def _distance_to_fig1b(wl):
    """Total variation distance between the tau_h distribution of `wl` (bins
    1..99 and the mass at >= 100, halting or not) and Fig. 1b's."""
    from tests.helpers import oracle_state
    c, long_, total = _fig1b()
    st, _ = oracle_state(wl, threads=os.cpu_count() or 1)
    t = st.steps[st.status == 1].astype(np.int64)
    q = np.bincount(t[t < 100], minlength=100)[:100].astype(float)
    ours = np.concatenate([q, [wl.num_vms - q.sum()]]) / wl.num_vms
    paper = np.concatenate([c, [long_]]) / total
    return 0.5 * np.abs(ours - paper).sum()


def test_fig1b_counts_and_the_distance_of_the_readings():
    """Fig. 1b's printed counts (8e6 programs, 3.36 % not halted within 10^6
    steps) against the sampler + lowering + oracle: the printed-rule reading
    is within about 0.2 in total variation, and fixing the output arity at 1
    (the App. B programs' arity) comes closer."""
    c, long_, total = _fig1b()
    assert abs(total - 8e6) < 100 and abs(269104 / total - 0.0336) < 5e-5
    assert c[:5].sum() == 0 and c[5] == 15462 and c.argmax() == 6   # nothing below 5; tau = 6 the mode
    kw = dict(L=100, seed=6, w=32, n=250, ell=10, s=2, cap=10 ** 4)
    d_default = _distance_to_fig1b(S.halting_programs(50000, **kw))
    d_e1 = _distance_to_fig1b(S.halting_programs(50000, out_arity=1, **kw))
    assert 0.15 < d_default < 0.27, d_default
    assert d_e1 < d_default - 0.01, (d_e1, d_default)
