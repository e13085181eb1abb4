"""Host-side failure injection (no GPU needed, nothing reaches a GPU): with
RASP_FAULT_INJECT=alloc every device allocation of the library fails the way
a failed cudaMalloc would, and the calls report RASP_ENOMEM with a message;
without it the same calls pass validation."""
import numpy as np
import pytest

from paper_2604_12902_gb300 import rasp as R


def cfg():
    return R.rasp_config(64, 0, 4, 8, 0, 0, 0, 0, 0, 0, None, None, 0)


def test_batch_create_reports_enomem(monkeypatch):
    monkeypatch.setenv("RASP_FAULT_INJECT", "alloc")
    with pytest.raises(R.RaspError) as e:
        R.rasp_batch_create(cfg(), np.full(16, 64, np.uint32))
    assert e.value.code == R.RASP_ENOMEM
    assert "injected" in R.rasp_last_error()


def test_pool_create_reports_enomem(monkeypatch):
    from paper_2604_12902_gb300 import serving as S
    monkeypatch.setenv("RASP_FAULT_INJECT", "alloc")
    with pytest.raises(R.RaspError) as e:
        S.Pool(1 << 20, 4, 8)
    assert e.value.code == R.RASP_ENOMEM


def test_validation_still_comes_first(monkeypatch):
    monkeypatch.setenv("RASP_FAULT_INJECT", "alloc")
    with pytest.raises(R.RaspError) as e:
        R.rasp_batch_create(cfg(), np.array([64, 0], np.uint32))     # n = 0 is invalid
    assert e.value.code == R.RASP_EINVAL
    monkeypatch.setenv("RASP_FAULT_INJECT", "none")
    assert R.rasp_batch_bytes(cfg(), np.full(16, 64, np.uint32)) > 0
