"""The C ABI from plain C: tests/c/rasp_client.c is compiled with gcc against
include/rasp.h and linked to librasp_gb300.so. Without a GPU it runs the
argument checks; with one it runs batches handed over in a binary file, and
its final state must equal the oracle's."""
import os
import subprocess

import numpy as np
import pytest

from paper_2604_12902_gb300 import workloads as W
from tests.helpers import assert_same_state, oracle_state

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    from paper_2604_12902_gb300 import build
    lib = build.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path_factory.mktemp("c") / "rasp_client")
    cmd = ["gcc", "-std=c11", "-O1", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "rasp_client.c"), "-o", exe,
           "-L", libdir, "-lrasp_gb300", "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_client_argument_checks_without_gpu(client):
    r = subprocess.run([client, "--no-gpu"], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert r.stdout.startswith("rasp_gb300")


def write_batch(path, wl, flags=0):
    progs, po = wl.expanded_programs()
    V = wl.num_vms
    with open(path, "wb") as f:
        np.array([V, progs.shape[0], wl.tapes.shape[0], wl.ell, wl.s, wl.w, flags], "<u8").tofile(f)
        np.asarray(wl.mem_words, "<u4").tofile(f)
        np.asarray(progs, "<i8").tofile(f)
        np.asarray(po, "<u8").tofile(f)
        np.asarray(wl.tapes, "<i8").tofile(f)
        np.asarray(wl.tape_off, "<u8").tofile(f)
        np.asarray(wl.caps, "<u8").tofile(f)


def read_state(path, wl):
    V, s = wl.num_vms, wl.s
    total = int(wl.mem_words.astype(np.uint64).sum())
    buf = open(path, "rb").read()
    o = 0
    out = {}
    for key, dt, count in (("i", "<i8", V), ("a", "<i8", V), ("steps", "<u8", V), ("status", "u1", V),
                           ("uhead", "<u4", V), ("ylen", "<u4", V), ("y", "<i8", V * s), ("mem", "<i8", total)):
        a = np.frombuffer(buf, dt, count, o)
        o += a.nbytes
        out[key] = a
    assert o == len(buf)
    out["y"] = out["y"].reshape(V, s)
    return out


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["random", "templates_w16", "ragged_plain"])
def test_c_client_runs_batches_like_the_oracle(client, tmp_path, case):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    flags = 0
    if case == "random":
        wl = W.random_programs(num_vms=3000, seed=11)
    elif case == "templates_w16":
        wl = W.template_programs(num_vms=2048, seed=12)
        wl.w = 16
    else:
        wl = W.uneven_programs(num_vms=4096, seed=13, n_hi=1024, cap_hi=4096)
        flags = 0x10                              # RASP_SCHED_PLAIN
    st, _ = oracle_state(wl, threads=os.cpu_count() or 1)
    src, dst = tmp_path / "in.bin", tmp_path / "out.bin"
    write_batch(src, wl, flags)
    r = subprocess.run([client, str(src), str(dst)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert_same_state(read_state(dst, wl), st, wl.ell, wl.s, what="C client " + case)


def test_header_compiles_and_links_from_cpp(tmp_path):
    """include/rasp.h is usable from C++ (extern "C" linkage) without a GPU."""
    from paper_2604_12902_gb300 import build
    libdir = os.path.dirname(build.build())
    src = tmp_path / "client.cpp"
    src.write_text('#include "rasp.h"\n#include <cstdio>\n#include <cstring>\n'
                   'int main() {\n'
                   '  rasp_config cfg; std::memset(&cfg, 0, sizeof cfg); cfg.word_bits = 1;\n'
                   '  uint32_t n[1] = {8}; uint64_t bytes = 0;\n'
                   '  if (rasp_batch_bytes(&cfg, 1, n, &bytes) != RASP_EINVAL) return 1;\n'
                   '  std::printf("%s\\n", rasp_version());\n  return 0;\n}\n')
    exe = str(tmp_path / "client")
    r = subprocess.run(["g++", "-std=c++11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-o", exe, "-L", libdir, "-lrasp_gb300", "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("rasp_gb300")
