"""bench.py's reference arm runs the CPU oracle (no GPU) and prints one JSON
line with the keys the benchmark contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "random",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_outcomes_reports_the_realised_timeout_rate():
    import bench
    o = bench.outcomes(dict(vm_steps=9, running=1, halted=6, timeout=3, fault_overflow=0, fault_addr=0))
    assert o["timeout"] == 3 and o["halted"] == 6 and abs(o["timeout_frac"] - 0.3) < 1e-12
    assert bench.outcomes(dict(running=0, halted=0, timeout=0, fault_overflow=0, fault_addr=0))["timeout_frac"] == 0.0


def test_clock_summary_from_nvidia_smi_lines():
    import bench
    lines = ["0, 2070, 2070, 812.40, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2070, 1390.02, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 1101.7, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "0, [N/A], 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active",   # unreadable sample
             "garbage"]
    c = bench.summarize_clocks(lines)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert bench.summarize_clocks([]) is None
    hot = bench.summarize_clocks(["0, 1500, 2070, 1400, 0x48, Active, Not Active, Active, Not Active"])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_algorithmic_bytes_per_opcode():
    """Bytes of VM state per executed step: 16 for the instruction fetch, 8
    more for an M operand read or write, 16 more for RD (tape read and M
    write) and PRI with room in y (M read and y write), 8 for PRI on a full
    y; the shared-program kernel fetches instructions from shared memory."""
    import bench
    ops = [0, 10, 20, 30, 40, 50, 60, 70]                 # LOD ADD MUL STO BNZ RD PRI
    st = dict(op_steps=ops, pri_full=5)
    want = 16 * 10 + 24 * 20 + 24 * 30 + 24 * 40 + 16 * 50 + 32 * 60 + 32 * 65 + 24 * 5
    assert bench.algorithmic_bytes(st) == want
    assert bench.algorithmic_bytes(st, fetch_from_smem=True) == want - 16 * sum(ops)


def test_program_words_go_up_as_int32_only_when_every_word_fits():
    """bench.py uploads programs through rasp_load_programs_i32 only when
    every word lies in [-2^31, 2^31) (the int32 values then stand for the
    same int64 words); the run kernel name follows the autotuner's report."""
    import numpy as np
    import bench
    from paper_2604_12902_gb300 import workloads as W
    wl = W.template_programs(num_vms=64, seed=2)
    assert bench.programs_fit_int32(wl)
    assert np.array_equal(wl.programs.astype(np.int32).astype(np.int64), wl.programs)
    for big in (1 << 31, -(1 << 31) - 1):
        wl2 = W.template_programs(num_vms=64, seed=2)
        wl2.programs = wl2.programs.copy()
        wl2.programs[1] = big
        assert not bench.programs_fit_int32(wl2)
    wl3 = W.template_programs(num_vms=64, seed=2)
    wl3.programs = wl3.programs.copy()
    wl3.programs[1], wl3.programs[3] = (1 << 31) - 1, -(1 << 31)
    assert bench.programs_fit_int32(wl3)
    assert bench.run_kernel_name("persist_smem e32 w1 step", 0) == "k_persist"
    assert bench.run_kernel_name("persist_gl e256 w4", 0) == "k_persist_gl"
    assert bench.run_kernel_name("shared", 0x20000) == "k_shared"
