"""Host-side checks of the allocation-free binding: a buffer of the wrong type, size,
layout or device raises before the library is called (no launch, no device access)."""
import pytest
import torch

from paper_2308_15407_gb300 import fdlb as F


@pytest.fixture
def no_library(monkeypatch):
    def fail():
        raise AssertionError("the library was reached")
    monkeypatch.setattr(F, "load", fail)


P64 = F.Params(nx=45, qx_half=6, qy=6, qz=0, kn=0.1, eta0=0.2, precision="fp64")
P32 = F.Params(nx=45, qx_half=6, qy=6, qz=0, kn=0.1, eta0=0.2, precision="fp32")


def test_f_elements_layout():
    # K = 2 Q x 2 Qy (2D reduced), rows padded to 64 nodes
    assert F.noalloc_f_elements(P64) == 12 * 12 * 64


@pytest.mark.parametrize("case", ["f_dtype", "f_size", "f_strided", "m_dtype", "m_short", "cpu", "two_phase"])
def test_bad_buffers_raise_before_the_library(no_library, case):
    n = F.noalloc_f_elements(P64)
    f = torch.zeros(n, dtype=torch.float64)
    m = torch.zeros(8 * P64.nx, dtype=torch.float64)
    p = P64
    if case == "f_dtype":
        f = f.float()
    elif case == "f_size":
        f = torch.zeros(n - 1, dtype=torch.float64)
    elif case == "f_strided":
        f = torch.zeros(2 * n, dtype=torch.float64)[::2]
    elif case == "m_dtype":
        m = m.float()
    elif case == "m_short":
        m = torch.zeros(8 * P64.nx - 1, dtype=torch.float64)
    elif case == "two_phase":
        p = F.Params(**{**P64.__dict__, "precision": "fp32+fp64"})
    with pytest.raises(ValueError):
        F.step_noalloc(p, f, 1, m)


def test_fp32_instance_needs_float32(no_library):
    f = torch.zeros(F.noalloc_f_elements(P32), dtype=torch.float64)
    with pytest.raises(ValueError, match="float32"):
        F.step_noalloc(P32, f, 1)
