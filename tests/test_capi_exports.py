"""The C-ABI library builds, loads without a GPU and exports every function
declared in include/rasp.h (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rasp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(rasp_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_function():
    from paper_2604_12902_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 13, names
    for name in names:
        assert hasattr(lib, name), name
    from paper_2604_12902_gb300 import rasp
    assert set(rasp.EXPORTS) <= set(names)


def test_batch_bytes_validates_without_gpu():
    from paper_2604_12902_gb300 import rasp
    import numpy as np
    cfg = rasp.rasp_config(64, 0, 4, 8, 0, 0, 0, 0, 0, 0, None, None, 0)
    nbytes = rasp.rasp_batch_bytes(cfg, np.full(1024, 64, np.uint32))
    assert nbytes > 1024 * 64 * 8 * 2
    cfg.word_bits = 1
    try:
        rasp.rasp_batch_bytes(cfg, np.full(4, 64, np.uint32))
        raise AssertionError("w = 1 must be rejected")
    except rasp.RaspError as e:
        assert e.code == rasp.RASP_EINVAL
    assert "version" not in rasp.rasp_last_error()
    assert rasp.rasp_version().startswith("rasp_gb300")


def test_narrow_batches_take_half_the_memory_words():
    """w <= 32 holds M in 4-byte words (plain and HBM-slab schedules); the
    shared-program and SMEM-staged schedules keep 8-byte words."""
    from paper_2604_12902_gb300 import rasp
    import numpy as np
    n = np.full(4096, 256, np.uint32)
    size = lambda w, flags: rasp.rasp_batch_bytes(rasp.rasp_config(w, 0, 4, 8, flags, 0, 0, 0, 0, 0, None, None, 0), n)
    m_words = 4096 * 256
    assert size(64, 0) - size(32, 0) >= 4 * m_words - 4096
    assert size(32, 0x10) == size(32, 0)
    assert size(32, 0x40) == size(64, 0x40) == size(64, 0)
    assert size(32, 0x20) == size(64, 0)
