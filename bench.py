"""Benchmark: VM-steps/s of the batched word RASP on GB300.

Workload (default): 1,048,576 template programs of 64 instructions (straight-
line arithmetic plus 1..3 counter-bounded loops, trips U[1,64]), n = 256
int64 words, 16-word input tapes U[-1000,1000], step cap 4096, seed 2.

One timed step = re-pack c_0 for every VM from the device-resident programs
and tapes (k_pack) + rasp_run to completion (k_persist): the whole hot path
on inputs already in HBM. M alone is 2 GiB, far larger than L2, so no flush is
needed between steps. `e2e` times the same work through the C ABI with host
buffers: rasp_load_programs + rasp_load_inputs from pinned host memory,
rasp_run, rasp_read_state of the per-VM results (i, a, steps, status, heads,
y). `roofline` rates the persistent kernel's algorithmic bytes (bytes of VM
state each executed opcode touches, weighted by the measured opcode mix)
against the measured HBM copy bandwidth. `cpu_baseline` is the serial C
oracle on a time-bounded prefix of the same workload.

Multi-GPU (torchrun): every rank runs its own disjoint 2^20-VM shard (no
collective on the data path); value = all ranks' steps / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "VM-steps/sec on 1 GB300 (and % of HBM roofline) vs plain form and CPU oracle"
UNIT = "VM-steps/s"
# bytes of VM state touched per executed step, by opcode (fetch 16 B; an M
# operand read or write 8 B; RD reads a tape word and writes M; PRI reads M
# and, when y has room, writes y)
BYTES_PER_OP = {1: 16, 2: 24, 3: 24, 4: 24, 5: 16, 6: 32, 7: 32}
PRI_FULL_BYTES = 24


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return summarize_clocks(self.lines)


def summarize_clocks(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen, from
    `nvidia-smi --query-gpu=<ClockSampler.Q> --format=csv,noheader,nounits`
    lines; None without a usable sample."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
        except ValueError:
            continue
        for k, nm in enumerate(names):
            if parts[5 + k].lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
            "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(name: str, rank: int, vms: int = 1 << 20, out_arity: int = 0):
    from paper_2604_12902_gb300 import workloads as W
    from paper_2604_12902_gb300.shards import shard_range
    if name == "templates":
        first, count = shard_range(rank, vms)
        return W.template_programs(num_vms=count, seed=2, first_vm=first), \
            "%s template programs (64 instr, 1-3 loops, trips U[1,64]), n=256, l=16, s=8, cap 4096" % format(vms, ",")
    if name == "uneven":
        wl = W.uneven_programs(num_vms=vms if vms != 1 << 20 else 1 << 22, seed=3,
                               first_vm=rank * (1 << 22), workers=os.cpu_count() or 1)
        return wl, ("%s uneven programs (length log-U[8,512], n log-U[16,4096], cap log-U[64,65536], "
                    "15%% built never to halt, ~33%% time out), l=16, s=8" % format(wl.num_vms, ","))
    if name == "shared":
        progs = 16384 if vms == 1 << 20 else max(1, vms // 256)    # --vms scales the number of programs
        wl = W.shared_programs(num_programs=progs)
        return wl, ("%s programs (48 instr, loop templates) x 256 tapes of 8 ints U[-50,50] = %s VMs, "
                    "n = 96 program + 128 data words, cap 2048" % (format(progs, ","), format(wl.num_vms, ",")))
    if name == "halting":
        from paper_2604_12902_gb300 import sampler as S
        first, count = shard_range(rank, vms)
        wl = S.halting_programs_parallel(count, workers=os.cpu_count() or 1, L=100, seed=6, cap=10 ** 6,
                                         first=first, out_arity=out_arity)
        return wl, ("%s programs of the array language, uniform over valid snippets of L = 100 tokens, "
                    "lowered (Sec. 2.2), w = 32, n = 250, l = 10, s = 2, tau_max = 10^6 (Sec. 3)%s"
                    % (format(wl.num_vms, ","), ", output arity %d" % out_arity if out_arity else ""))
    if name == "random":
        return W.random_programs(num_vms=1024, seed=1, first_vm=rank * 1024), \
            "1,024 random programs (32 instr, opcodes U{1..7}, operands U[0,63]), n=64, l=4, s=8, cap 256"
    raise SystemExit("unknown workload %s" % name)


def profiled_traffic(vm_steps: int):
    """DRAM bytes of one run launch from the committed ncu measurement of the
    run kernel (`profiles/traffic.json`: bytes per VM-step of a captured small
    case, scaled by VM-steps), or None when a source file the kernel is built
    from changed since that capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)["k_persist_gl templates"]
        h = hashlib.sha256()
        for name in rec["sources"]:
            with open(os.path.join(ROOT, "paper_2604_12902_gb300", "csrc", name), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest() != rec["sources_sha256"]:
            return None
        return float(rec["dram_bytes_per_vm_step"]) * vm_steps
    except (OSError, KeyError, ValueError, TypeError):
        return None


def outcomes(stats) -> dict:
    """Final statuses of the batch after a step, with the realised timeout
    rate (the fraction of VMs stopped by their step cap)."""
    keys = ("halted", "timeout", "running", "fault_overflow", "fault_addr")
    out = {k: int(stats[k]) for k in keys}
    total = sum(out.values())
    out["timeout_frac"] = out["timeout"] / total if total else 0.0
    return out


def algorithmic_bytes(stats, fetch_from_smem: bool = False, word_bytes: int = 8) -> float:
    """Opcode-weighted bytes of VM state touched by the executed steps; with
    fetch_from_smem the 16-byte instruction fetch is left out (the
    shared-program kernel reads the program words from shared memory). The
    table is in 8-byte words; a batch held in 4-byte words (w <= 32) touches
    half as many bytes per access."""
    ops = stats["op_steps"]
    b = sum(BYTES_PER_OP[k] * ops[k] for k in range(1, 8))
    b -= (BYTES_PER_OP[7] - PRI_FULL_BYTES) * stats["pri_full"]
    if fetch_from_smem:
        b -= 16 * sum(ops[k] for k in range(1, 8))
    return float(b) * word_bytes / 8.0


KERNEL_OF = {"persist_gl": "k_persist_gl", "plain": "k_plain", "persist_smem": "k_persist", "shared": "k_shared_loop"}
SCHED_NAME = {0x10: "plain", 0x20: "persist_smem", 0x30: "persist_gl", 0x40: "shared"}


def run_kernel_name(chosen: str, flags: int) -> str:
    """The run kernel a schedule name (autotuner report) or flag set selects."""
    kernel = KERNEL_OF.get(chosen.split()[0], chosen)
    if kernel == "k_shared_loop" and flags & 0x20000:     # RASP_STEP_BLOCK: the one-step form
        kernel = "k_shared"
    return kernel


PROGRAM_WORDS = {True: "int32 (every program word fits; sign-extended on the device, machine words w bits)",
                 False: "int64"}


def programs_fit_int32(wl) -> bool:
    """Every program word fits in 32 bits (a signed int32)."""
    return bool(wl.programs.size) and int(wl.programs.min()) >= -(1 << 31) and int(wl.programs.max()) < (1 << 31)


def load_wl(R, b, wl, p32=None):
    """Load a workload into a batch; programs whose words all fit in 32 bits
    go through rasp_load_programs_i32 (p32: those words as int32), which
    keeps them as 4-byte words on the device where they fit beside M and
    sign-extends them in the pack. The machine words stay w bits."""
    if p32 is not None:
        R.rasp_load_programs_i32(b.h, p32, wl.prog_off, wl.prog_of_vm)
    else:
        b.load_programs(wl.programs, wl.prog_off, wl.prog_of_vm)
    b.load_inputs(wl.tapes, wl.tape_off, wl.caps)


def time_config(R, torch, wl, desc, flags, steps, warmup, flush_l2=False):
    """Times one workload the way the headline is timed (re-pack c_0 + run to
    completion per step, CUDA events on the batch stream, generation and
    tuning untimed): run-kernel ms, whole-step VM-steps/s, roofline of the
    run kernel against the measured HBM bandwidth, and the final statuses."""
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if flush_l2 else None
    p32 = wl.programs.astype(np.int32) if programs_fit_int32(wl) else None
    with R.Batch(wl.mem_words, wl.ell, wl.s, word_bits=wl.w, flags=flags) as b:
        load_wl(R, b, wl, p32)
        tuned = b.autotune(reps=2) if (flags & 0xF0) == 0 else None
        with R.Batch(wl.mem_words, wl.ell, wl.s, word_bits=wl.w, flags=flags | R.COLLECT_STATS) as bs:
            load_wl(R, bs, wl, p32)
            bs.run()
            stats = bs.stats()
        chosen = tuned["chosen"] if tuned else "flags %#x" % flags
        kernel = run_kernel_name(chosen if tuned else SCHED_NAME.get(flags & 0xF0, "persist_gl"), flags)
        word_bytes = b.describe().get("word_bytes", 8)
        alg = algorithmic_bytes(stats, fetch_from_smem=kernel.startswith("k_shared"), word_bytes=word_bytes)
        for _ in range(warmup):
            b.reset()
            b.run()
        torch.cuda.synchronize()
        run_ms, pack_ms, step_ms = [], [], []
        for _ in range(steps):
            if flush is not None:
                flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            b.reset()
            ev[1].record(stream)
            b.run()
            ev[2].record(stream)
            torch.cuda.synchronize()
            pack_ms.append(ev[0].elapsed_time(ev[1]))
            run_ms.append(ev[1].elapsed_time(ev[2]))
            step_ms.append(ev[0].elapsed_time(ev[2]))
        b.sync()
        st = b.stats()
    assert st["vm_steps"] == stats["vm_steps"], "timed runs disagree with the counting run"
    hbm, peak_kind = peaks()
    run_avg = float(np.mean(run_ms))
    achieved = alg / (run_avg * 1e-3) / 1e9
    m_bytes = float(wl.mem_words.astype(np.uint64).sum()) * 8.0
    return {"workload": desc, "vms": wl.num_vms, "vm_steps": int(stats["vm_steps"]), "steps": steps,
            "warmup": warmup, "ms_per_step": float(np.mean(step_ms)),
            "value": stats["vm_steps"] / (float(np.mean(step_ms)) * 1e-3), "unit": UNIT,
            "schedule": chosen, "cuda_graph": bool(flags & R.CUDA_GRAPH), "program_words": PROGRAM_WORDS[p32 is not None],
            "l2": ("inputs larger than L2 (M = %.2f GiB)" % (m_bytes / 2 ** 30)) if m_bytes > 129e6
            else ("M = %.2f MB fits in L2: 256 MB written between timed steps" % (m_bytes / 1e6)),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": None, "kernel": kernel, "peak_kind": peak_kind,
                         "bytes_per_step": alg / max(stats["vm_steps"], 1),
                         "fetch_from_smem_excluded": kernel.startswith("k_shared"), "word_bytes": word_bytes,
                         "kernel_ms": run_avg, "pack_ms": float(np.mean(pack_ms))},
            "outcomes": outcomes(st)}


def other_configs(R, torch, steps, warmup, serving=True):
    """The benchmark's other single-GPU configurations, each timed like the
    headline after it: 1,024 random programs (config 1), the uneven batch of
    4,194,304 programs in its CUDA-graph form (config 3), the shared-program
    rollout of 16,384 programs x 256 tapes (config 4), the halting workload of
    Sec. 3 (2^20 sampled programs, w = 32, tau_max = 10^6), and serving at 200
    requests/s for 60 s (config 5: p50/p99 latency and VM-steps/s)."""
    out = {}
    for name in ("random", "shared", "uneven", "halting"):
        t0 = time.perf_counter()
        wl, desc = make_workload(name, 0)
        gen_s = time.perf_counter() - t0
        # the halting workload (Sec. 3, w = 32) runs on the HBM-slab schedule
        # without autotuning (one plain-form trial alone takes 2.8 s)
        flags = R.CUDA_GRAPH if name == "uneven" else (R.SCHED_PERSIST_GL if name == "halting" else 0)
        clk = ClockSampler(torch.cuda.current_device())
        clk.start()
        rec = time_config(R, torch, wl, desc, flags, steps, warmup, flush_l2=name == "random")
        rec["clocks"] = clk.stop()
        rec["generation_s"] = gen_s
        out[{"random": "config1_random", "uneven": "config3_uneven", "shared": "config4_shared",
             "halting": "next2_halting"}[name]] = rec
        del wl
        torch.cuda.empty_cache()
    if not serving:
        return out
    # config 5: serving at 200 requests/s for 60 s (request generation untimed)
    m = serving_measure(torch, 200.0, 60.0)
    o = m["out"]
    out["config5_serving"] = {"workload": m["desc"], "lambda": 200.0, "duration_s": 60.0,
                              "requests_done": o["requests"], "p50_ms": o["p50_ms"], "p99_ms": o["p99_ms"],
                              "value": o["vm_steps_per_s"], "unit": UNIT, "vm_steps": o["vm_steps"],
                              "wall_s": o["wall_s"], "offered_vms_per_s": m["offered"],
                              "mean_vms_per_request": o["mean_vms"], "pool": m["pool"], "clocks": m["clocks"],
                              "generation_s": m["gen_s"]}
    torch.cuda.empty_cache()
    return out


def cpu_baseline(wl, budget_s: float = 15.0, threads: int = 1, classic: bool = False):
    """The serial oracle on a prefix of the workload, chunk by chunk until
    `budget_s` seconds have passed."""
    from oracle import oracle
    chunk = 8192
    done_vms, steps, t_used = 0, 0, 0.0
    while done_vms < wl.num_vms and t_used < budget_s:
        hi = min(wl.num_vms, done_vms + chunk)
        sub = wl.subset(np.arange(done_vms, hi))
        t0 = time.perf_counter()
        st, _ = oracle.run_packed(sub.programs, sub.prog_off, sub.mem_words, sub.tapes, sub.tape_off,
                                  sub.ell, sub.s, caps=sub.caps, w=sub.w, threads=threads, classic=classic)
        t_used += time.perf_counter() - t0
        steps += int(st.steps.sum())
        done_vms = hi
    return {"value": steps / t_used, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "first %d of %d VMs (%d VM-steps, pack+run, %.1f s)" % (done_vms, wl.num_vms, steps, t_used)}


def run_reference(args, ws, rank):
    """Reference arm: the CPU oracle as it stands, on bounded samples."""
    if rank != 0:
        return
    from oracle import oracle
    wl, desc = make_workload(args.workload, 0, out_arity=args.out_arity)
    threads = os.cpu_count() or 1
    sample = min(wl.num_vms, 1 << 16)
    sub = wl.subset(np.arange(sample))
    times, steps = [], 0
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        st, _ = oracle.run_packed(sub.programs, sub.prog_off, sub.mem_words, sub.tapes, sub.tape_off,
                                  sub.ell, sub.s, caps=sub.caps, w=sub.w, threads=threads,
                                  classic=args.isa == "classic")
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
            steps += int(st.steps.sum())
    value = steps / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": desc + " (first %d VMs per step)" % sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "first %d VMs, pack+run, %d threads" % (sample, threads)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serving_measure(torch, lam, duration, n_requests=64, arena_gb=192.0, lam_sweep=(), sweep_duration=10.0):
    """Config 5: open-loop Poisson arrivals of rollout requests (each 1k-100k
    programs drawn like the uneven batch) into one device arena; requests are
    admitted as memory frees up and run concurrently (continuous batching).
    Returns the run's figures, those of any further arrival rates, the
    clocks sampled during the main run and the pool's counters."""
    from paper_2604_12902_gb300 import serving as SV, workloads as W
    rng = np.random.default_rng(11)
    u = rng.integers(0, 1 << 32, size=n_requests, dtype=np.uint64).astype(np.uint32)
    sizes = W.log_uniform_int(u, 1000, 100000)
    t0 = time.perf_counter()
    reqs = [W.uneven_programs(num_vms=int(n), seed=5, first_vm=k * 100_000, workers=os.cpu_count() or 1)
            for k, n in enumerate(sizes)]
    gen_s = time.perf_counter() - t0
    for wl in reqs:     # requests arrive in page-locked host memory (async H2D)
        for f in ("programs", "prog_off", "tapes", "tape_off", "caps", "mem_words"):
            setattr(wl, f, _pinned_copy(torch, getattr(wl, f)))
    free, _ = torch.cuda.mem_get_info()
    arena = int(min(arena_gb * 2 ** 30, free * 0.8))
    sweep = []
    with SV.Pool(arena, reqs[0].ell, reqs[0].s) as pool:
        SV.poisson_run(pool, reqs[:4], lam=50.0, duration=0.2, seed=0)      # warm-up (untimed)
        clk = ClockSampler(torch.cuda.current_device())
        clk.start()
        out = SV.poisson_run(pool, reqs, lam=lam, duration=duration, seed=1)
        clocks = clk.stop()
        pool_counters = pool.stats()
        # higher arrival rates on the same requests: where does latency grow?
        for lam2 in lam_sweep:
            o = SV.poisson_run(pool, reqs, lam=lam2, duration=sweep_duration, seed=2, max_waiting=32)
            sweep.append({"lambda": lam2, "p50_ms": o["p50_ms"], "p99_ms": o["p99_ms"],
                          "vm_steps_per_s": o["vm_steps_per_s"], "requests_done": o["requests"],
                          "rejected": o["rejected"], "wall_s": o["wall_s"],
                          "offered_vms_per_s": lam2 * float(np.mean([r.num_vms for r in reqs]))})
    offered = lam * float(np.mean([r.num_vms for r in reqs]))
    desc = ("serving: Poisson arrivals (lambda %.0f/s) for %.0f s of rollout requests, each log-U[1e3,1e5] "
            "programs drawn as the uneven batch, inputs in pinned host memory; %d distinct requests cycled; "
            "arena %.1f GiB" % (lam, duration, len(reqs), arena / 2 ** 30))
    return {"out": out, "sweep": sweep, "clocks": clocks, "pool": pool_counters, "gen_s": gen_s,
            "offered": offered, "desc": desc}


def run_serving(args, ws, rank):
    import torch
    torch.cuda.set_device(0)
    m = serving_measure(torch, args.lam, args.duration, args.requests, args.arena_gb,
                        [float(x) for x in args.lam_sweep.split(",") if x], args.sweep_duration)
    out = m["out"]
    line = {"metric": METRIC, "value": out["vm_steps_per_s"], "unit": UNIT, "n_gpus": 1, "steps": out["requests"],
            "warmup": 1, "ms_per_step": out["wall_s"] * 1e3 / max(out["requests"], 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": m["desc"]},
            "serving": {"requests_done": out["requests"], "p50_ms": out["p50_ms"], "p99_ms": out["p99_ms"],
                        "wall_s": out["wall_s"], "vm_steps": out["vm_steps"], "mean_vms_per_request": out["mean_vms"],
                        "offered_vms_per_s": m["offered"], "request_gen_s": m["gen_s"], "lambda_sweep": m["sweep"],
                        "sweep_duration_s": args.sweep_duration, "pool": m["pool"],
                        "design": "one persistent serving kernel over a device ring shared by all admitted requests"},
            "clocks": m["clocks"]}
    print(json.dumps(line), flush=True)


def run_search(args):
    """Generate -> run -> filter (busy-beaver search): rounds of programs of
    L = 100 tokens drawn uniformly, run on the device to tau_max, the best
    halting programs kept by a device top-k; host generation of the next round
    overlaps the device run of the current one. Reported end to end."""
    import torch
    from paper_2604_12902_gb300 import search
    torch.cuda.set_device(0)
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    res = search.busy_beaver_search(args.rounds, args.vms, k=16, L=100, seed=6, tau_max=args.tau_max)
    clocks = clk.stop()
    line = {"metric": METRIC, "value": res["vm_steps"] / res["wall_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.rounds, "warmup": 0, "ms_per_step": res["wall_s"] * 1e3 / args.rounds,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": "busy-beaver search: %d rounds x %s programs of L = 100 tokens (uniform), w = 32, "
                                   "n = 250, tau_max = %d, device top-16 per round" % (args.rounds, format(args.vms, ","),
                                                                                    args.tau_max)},
            "search": {"programs": res["programs"], "programs_per_s": res["programs_per_s"], "halted": res["halted"],
                       "wall_s": res["wall_s"], "device_s": res["gpu_s"], "waiting_for_generation_s": res["gen_wait_s"],
                       "best": [{"tau_h": t, "program": pid, "source": src} for t, pid, src in res["best"][:4]]},
            "clocks": clocks}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="templates", choices=["templates", "uneven", "shared", "random", "serving", "halting", "search"])
    ap.add_argument("--flags", type=lambda x: int(x, 0), default=0, help="rasp_config.flags (schedule)")
    ap.add_argument("--isa", default="word", choices=["word", "classic"],
                    help="opcode set: the word machine (Sec. 2.1) or the classic one (Sec. 1.1: SUB, BPA)")
    ap.add_argument("--epoch", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="resident CTAs per SM of the persistent kernels (0: as many as fit)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the (untimed) schedule autotuning")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--vms", type=int, default=1 << 20, help="template programs per GPU (profiling cases)")
    ap.add_argument("--lam", type=float, default=200.0, help="serving: arrival rate (requests/s)")
    ap.add_argument("--duration", type=float, default=60.0, help="serving: seconds of arrivals")
    ap.add_argument("--requests", type=int, default=64, help="serving: distinct requests (cycled)")
    ap.add_argument("--arena-gb", type=float, default=192.0, help="serving: device arena size (at most 80%% of free memory)")
    ap.add_argument("--lam-sweep", default="", help="serving: further arrival rates to run, comma separated")
    ap.add_argument("--sweep-duration", type=float, default=10.0, help="serving: seconds of arrivals per swept rate")
    ap.add_argument("--rounds", type=int, default=4, help="search: rounds")
    ap.add_argument("--tau-max", type=int, default=10 ** 5, help="search: step cap")
    ap.add_argument("--no-serving", action="store_true",
                    help="leave config 5 (60 s of serving) out of the other configurations")
    ap.add_argument("--e2e-batches", type=int, default=3,
                    help="end-to-end leg: batches in flight (each on a stream of its own)")
    ap.add_argument("--no-other", action="store_true",
                    help="skip the other configurations (random, uneven, shared) after the headline")
    ap.add_argument("--out-arity", type=int, default=0,
                    help="halting: output arity of the sampled programs (0 = drawn from 1..s, as the grammar allows)")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload == "serving":
        if rank == 0:
            run_serving(args, ws, rank)
        return
    if args.workload == "search":
        if rank == 0:
            run_search(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2604_12902_gb300 import rasp as R
    from paper_2604_12902_gb300.shards import combine
    if args.isa == "classic":
        args.flags |= R.ISA_CLASSIC

    wl, desc = make_workload(args.workload, rank, args.vms, args.out_arity)
    stream = torch.cuda.current_stream()
    b = R.Batch(wl.mem_words, wl.ell, wl.s, word_bits=wl.w, flags=args.flags, epoch=args.epoch,
                ctas_per_sm=args.ctas_per_sm)
    p32 = wl.programs.astype(np.int32) if programs_fit_int32(wl) else None
    load_wl(R, b, wl, p32)
    tuned = None
    if (args.flags & R.SCHED_PERSIST_GL) == 0 and not args.epoch and not args.ctas_per_sm and not args.no_tune:
        tuned = b.autotune(reps=2)      # untimed: measured schedule choice, state unchanged

    # opcode mix (and total steps) from an untimed counting run
    with R.Batch(wl.mem_words, wl.ell, wl.s, word_bits=wl.w, flags=args.flags | R.COLLECT_STATS, epoch=args.epoch) as bs:
        load_wl(R, bs, wl, p32)
        bs.run()
        stats = bs.stats()
    total_steps = stats["vm_steps"]
    kernel = run_kernel_name(tuned["chosen"] if tuned else SCHED_NAME.get(args.flags & 0xF0, "persist_gl"), args.flags)
    # the shared-program kernel reads instruction pairs from shared memory
    word_bytes = b.describe().get("word_bytes", 8)
    alg_bytes = algorithmic_bytes(stats, fetch_from_smem=kernel.startswith("k_shared"), word_bytes=word_bytes)

    # halting workload: the tau_h histogram is computed on the device in every step
    hist_edges = np.concatenate([np.arange(0, 101), [10 ** 6, 1 << 62]]).astype(np.uint64)
    hist = {}

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        b.reset()
        if evs:
            evs[1].record(stream)
        b.run()
        if evs:
            evs[2].record(stream)
        if args.workload == "halting":
            hist["counts"], hist["other"] = b.halting_histogram(hist_edges)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    run_ms = [e[1].elapsed_time(e[2]) for e in evs]
    pack_ms = [e[0].elapsed_time(e[1]) for e in evs]
    b.sync()
    st = b.stats()
    run_launches = int(st["launches"])
    m_bytes = float(wl.mem_words.astype(np.uint64).sum()) * 8.0
    assert st["vm_steps"] == total_steps, "timed runs disagree with the counting run"

    ms_total, steps_total = combine(dist, elapsed_ms, total_steps, device="cuda")
    ms_per_step = ms_total / args.steps
    value = steps_total / (ms_per_step * 1e-3)

    hbm, peak_kind = peaks()
    run_avg = float(np.mean(run_ms))
    achieved = alg_bytes / (run_avg * 1e-3) / 1e9
    # the summary was taken on the default launch shape (HBM-slab persistent,
    # 4 warps x 7 CTAs per SM, epoch 128); a tuned shape that differs only in
    # its epoch runs the same kernel at the same occupancy
    chosen = tuned.get("chosen", "") if tuned else "persist_gl e128 w4"
    same_shape = args.workload == "templates" and args.flags == 0 and not args.epoch and \
        chosen.startswith("persist_gl e") and chosen.endswith(" w4")
    traffic = profiled_traffic(total_steps) if same_shape else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic,
                "traffic_source": "profiles/traffic.json (ncu, 262,144-VM case, epoch 128, scaled by VM-steps)"
                if traffic is not None else None,
                "kernel": kernel, "peak_kind": peak_kind,
                "fetch_from_smem_excluded": kernel.startswith("k_shared"), "word_bytes": word_bytes,
                "bytes_per_step": alg_bytes / max(total_steps, 1),
                "kernel_ms": run_avg, "pack_ms": float(np.mean(pack_ms))}

    # plain one-launch-per-batch form on the same workload (untimed by the contract)
    plain = None
    if not args.no_plain:
        with R.Batch(wl.mem_words, wl.ell, wl.s, word_bits=wl.w, flags=R.SCHED_PLAIN | (args.flags & R.ISA_CLASSIC)) as bp:
            bp.load_workload(wl)
            bp.run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ts = []
            for _ in range(3):
                bp.reset()
                e0.record(stream)
                bp.run()
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            plain = {"value": total_steps / (np.median(ts) * 1e-3), "unit": UNIT, "kernel_ms": float(np.median(ts)),
                     "persistent_speedup": float(np.median(ts)) / run_avg}

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        pin = lambda a: _pinned_copy(torch, a)
        # programs whose words all fit in 32 bits go up as int32 words (half
        # the bytes; the library sign-extends them on the device)
        narrow_prog = p32 is not None
        h_prog = pin(p32 if narrow_prog else wl.programs)
        h_poff = pin(wl.prog_off)
        load_programs = R.rasp_load_programs_i32 if narrow_prog else R.rasp_load_programs
        h_pvm = pin(wl.prog_of_vm) if wl.prog_of_vm is not None else None
        h_tape, h_toff, h_caps = pin(wl.tapes), pin(wl.tape_off), pin(wl.caps)
        out = {k: pin(np.empty(wl.num_vms, dt)) for k, dt in
               (("i", np.int64), ("a", np.int64), ("steps", np.uint64), ("status", np.uint8),
                ("uhead", np.uint32), ("ylen", np.uint32))}
        out["y"] = pin(np.empty(wl.num_vms * wl.s, np.int64))
        h2d = sum(x.nbytes for x in (h_prog, h_poff, h_tape, h_toff, h_caps) + ((h_pvm,) if h_pvm is not None else ()))
        d2h = sum(x.nbytes for x in out.values())

        # NB batches in flight (default 3): step t uploads, packs and runs
        # batch t % NB while the runs of earlier steps finish on their own
        # streams; a second host thread reads each step's results back as
        # soon as its run is done, so that reads (device to host) overlap
        # uploads (host to device). A batch is loaded again only after its
        # previous results have been read: with two batches the upload of
        # step t waits for the read of step t - 2, which ends one read after
        # the run before it, so upload + read + host work must fit in one
        # run; a third batch gives them two. Every step still copies its own
        # inputs host -> device and its results device -> host inside the
        # timed region.
        from concurrent.futures import ThreadPoolExecutor
        plan = b.describe()["buckets"][0]
        sched = {"plain": R.SCHED_PLAIN, "persist": R.SCHED_PERSIST, "persist_gl": R.SCHED_PERSIST_GL,
                 "shared": R.SCHED_SHARED}[plan["schedule"]]
        # each batch on a stream of its own (not the legacy default stream,
        # which would order every other stream's work around its own)
        nb = max(1, args.e2e_batches)
        e2e_streams = [torch.cuda.Stream() for _ in range(nb)]
        pair = [R.Batch(wl.mem_words, wl.ell, wl.s, word_bits=wl.w, flags=(args.flags & ~0xF0) | sched,
                        epoch=plan["epoch"], warps_per_cta=plan["warps_per_cta"], ctas_per_sm=plan["ctas_per_sm"],
                        stream=e2e_streams[k].cuda_stream) for k in range(nb)]
        outs = [out] + [{k: pin(np.empty_like(v)) for k, v in out.items()} for _ in range(nb - 1)]
        views = [R.rasp_state_view(*(R._p(o[k]) for k in ("i", "a", "steps", "status", "uhead", "ylen", "y")),
                                   None, 0) for o in outs]
        reader = ThreadPoolExecutor(1)
        reads = [None] * nb

        def e2e_step(t):
            x = t % nb
            if reads[x] is not None:
                reads[x].result()            # batch x's previous results are out before it is reloaded
            # inputs first: their load queues no kernel, so that neither load's
            # wait for its host copies stalls behind the other batch's run
            R.rasp_load_inputs(pair[x].h, h_tape, h_toff, h_caps)
            load_programs(pair[x].h, h_prog, h_poff, h_pvm)
            R.rasp_run(pair[x].h)
            reads[x] = reader.submit(R.rasp_read_state, pair[x].h, 0, wl.num_vms, views[x])

        def e2e_drain():
            for x in range(nb):
                if reads[x] is not None:
                    reads[x].result()
                    reads[x] = None

        for t in range(max(4, 2 * nb)):
            e2e_step(t)
        e2e_drain()
        torch.cuda.synchronize()
        n_e2e = max(4, 2 * nb, args.steps)
        t0 = time.perf_counter()
        for t in range(n_e2e):
            e2e_step(t)
        e2e_drain()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / n_e2e
        reader.shutdown()
        # the copy engines' host-to-device rate on this machine, for context:
        # one copy of the program words from pinned memory, timed alone
        dbuf = torch.empty(h_prog.nbytes, dtype=torch.uint8, device="cuda")
        hsrc = torch.from_numpy(h_prog.view(np.uint8).reshape(-1))
        dbuf.copy_(hsrc, non_blocking=True)
        torch.cuda.synchronize()
        tc = time.perf_counter()
        dbuf.copy_(hsrc, non_blocking=True)
        torch.cuda.synchronize()
        h2d_gbs = h_prog.nbytes / (time.perf_counter() - tc) / 1e9
        del dbuf
        for o in outs:
            assert int(o["steps"].sum()) == total_steps
        for x in pair:
            x.close()
        e2e_val = total_steps / dt
        if dist:
            t_max, _ = combine(dist, dt, total_steps, device="cuda")
            e2e_val = steps_total / t_max
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": dt * 1e3, "steps": n_e2e, "h2d_gbs_alone": h2d_gbs,
               "program_words": PROGRAM_WORDS[narrow_prog],
               "pipeline": "%d batches in flight, each on a stream of its own, results read back by a second "
                           "host thread: uploads overlap earlier steps' runs and read-backs" % nb}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(wl, args.cpu_seconds, classic=args.isa == "classic")
    b.close()
    num_vms = wl.num_vms
    del wl
    torch.cuda.empty_cache()

    # the other configurations, after the headline has been timed
    others = None
    if rank == 0 and ws == 1 and args.workload == "templates" and args.vms == 1 << 20 and args.flags == 0 \
            and not args.no_other:
        others = other_configs(R, torch, args.steps, args.warmup, serving=not args.no_serving)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": {"workload": desc, "vms_per_gpu": num_vms, "vm_steps_per_gpu": total_steps,
                           "l2": "inputs larger than L2 (M = %.2f GiB)" % (m_bytes / 2 ** 30)
                                 if m_bytes > 129e6 else "M below L2 size (%.1f MB); no flush" % (m_bytes / 1e6),
                           "schedule_flags": args.flags, "isa": args.isa, "parallelism": "vm shards x%d" % ws,
                           "schedule": tuned["chosen"] if tuned else "flags %#x" % args.flags,
                           "program_words": PROGRAM_WORDS[p32 is not None]},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "plain": plain,
                "gpu_launches": (1 + run_launches + (1 if hist else 0)) * args.steps, "clocks": clocks,
                "outcomes": outcomes(st)}
        if others:
            line["other_configs"] = others
        if hist:
            c, o = hist["counts"], hist["other"]
            halted = int(c.sum() + o[3])
            line["halting"] = {
                "programs": num_vms, "halted": halted, "halted_frac": halted / num_vms,
                "tau_h_lt_100": int(c[:100].sum()), "tau_h_100_to_1e6": int(c[100]), "timeout_1e6": int(o[1]),
                "mean_tau_h_lt_100": float((c[:100] * np.arange(100)).sum() / max(c[:100].sum(), 1)),
                "min_tau_h": int(np.nonzero(c)[0][0]) if c.any() else None,
                "wall_s_per_run": run_avg * 1e-3,
                "paper_context": "Fig. 1: 8e6 programs (its own sampler), 96.6 % halt, 211 with tau_h in "
                                 "[100, 1e6), mean tau_h ~18.2; 1x B200 1.1 s for 1e6 programs"}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


_PINNED = []


def _pinned_copy(torch, a):
    """A copy of `a` in page-locked host memory (kept alive for the run)."""
    t = torch.empty(max(a.nbytes, 1), dtype=torch.uint8, pin_memory=True)
    _PINNED.append(t)
    arr = t.numpy()[: a.nbytes].view(a.dtype).reshape(a.shape)
    arr[...] = a
    return arr


if __name__ == "__main__":
    main()
