"""C-ABI checks that need no GPU: the library loads, exports every symbol include/fdlb.h
declares, validates parameters, and its host-side Gauss rules match the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import quadrature as qd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fdlb.h")


@pytest.fixture(scope="module")
def F():
    from paper_2308_15407_gb300 import fdlb
    if not os.path.exists(fdlb.LIB_PATH):
        from paper_2308_15407_gb300 import build
        build.build()
    return fdlb


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fdlb_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(F):
    lib = ctypes.CDLL(F.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_abi_version_and_struct(F):
    lib = F.load()
    hdr = open(os.path.join(ROOT, "include", "fdlb.h")).read()
    assert lib.fdlb_abi_version() == int(re.search(r"#define FDLB_ABI_VERSION (\d+)", hdr).group(1))
    assert ctypes.sizeof(F.CParams) == 4 * 11 + 4 + 8 * 11        # 11 int32, padding, 11 doubles


def test_parameter_validation(F):
    ok = F.Params(nx=50, qx_half=4, qy=4, qz=4, kn=0.1, eta0=0.1)
    assert F.workspace_bytes([ok]) > 0
    bad = [dict(nx=4), dict(qx_half=0), dict(qx_half=101), dict(qy=1), dict(qz=2), dict(qy=0, qz=4),
           dict(eta0=0.5), dict(kn=0.0), dict(T_left=0.0), dict(qy=0, qz=0, U_left=0.1)]
    for kw in bad:
        p = F.Params(**{**ok.__dict__, **kw})
        with pytest.raises(F.FdlbError):
            F.workspace_bytes([p])
    c = ok.to_c()
    c.struct_size = 8
    lib = F.load()
    assert lib.fdlb_workspace_bytes((F.CParams * 1)(c), 1) == 0
    assert b"struct_size" in lib.fdlb_last_error(None)


def test_chi_model_validation(F):
    """RET-FM instances carry their averaging weights; unknown models and eta0 = 0 are rejected."""
    base = dict(nx=64, qx_half=4, qy=0, qz=0, kn=0.05, eta0=0.1)
    b_set = F.workspace_bytes([F.Params(**base)])
    b_fm = F.workspace_bytes([F.Params(**base, chi_model="ret-fm")])
    assert b_fm > b_set
    lib = F.load()
    c = F.Params(**base).to_c()
    c.chi_model = 2
    assert lib.fdlb_workspace_bytes((F.CParams * 1)(c), 1) == 0
    assert b"chi_model" in lib.fdlb_last_error(None)
    with pytest.raises(F.FdlbError):
        F.workspace_bytes([F.Params(**{**base, "eta0": 0.0}, chi_model="ret-fm")])


def test_null_context_calls_fail_cleanly(F):
    """Calls on a null context return FDLB_EINVAL without touching a device."""
    lib = F.load()
    out = np.zeros(4)
    assert lib.fdlb_residual(None, F._dptr(out)) == F.FDLB_EINVAL
    assert b"fdlb_residual" in lib.fdlb_last_error(None)
    assert lib.fdlb_status(None, F._dptr(out), None, None) == F.FDLB_EINVAL
    assert lib.fdlb_step(None, 1, 0.0) == F.FDLB_EINVAL


def test_x_quadrature_validation(F):
    """Orders: half-range up to 100 per side (Table 1 of Sec. IV reaches 29; the mass flow above
    Kn = 1 uses 100), full-range up to 200 (App. A's comparison needs ~200); the full rule's
    tables hold 2 qx_half polynomials."""
    base = dict(nx=64, qx_half=8, qy=4, qz=0, kn=0.1, eta0=0.1)
    b_half = F.workspace_bytes([F.Params(**base)])
    b_full = F.workspace_bytes([F.Params(**base, x_quadrature="full")])
    assert b_full > b_half                      # w_k h_l(p_k) for l < 16 instead of l < 8
    assert F.workspace_bytes([F.Params(**{**base, "qx_half": 100}, x_quadrature="full")]) > 0
    with pytest.raises(F.FdlbError):
        F.workspace_bytes([F.Params(**{**base, "qx_half": 101}, x_quadrature="full")])
    assert F.workspace_bytes([F.Params(**{**base, "qx_half": 100})]) > 0
    with pytest.raises(F.FdlbError):
        F.workspace_bytes([F.Params(**{**base, "qx_half": 101})])
    lib = F.load()
    c = F.Params(**base).to_c()
    c.x_quadrature = 2
    assert lib.fdlb_workspace_bytes((F.CParams * 1)(c), 1) == 0
    assert b"x_quadrature" in lib.fdlb_last_error(None)


def test_two_phase_precision_workspace(F):
    """FP32-then-FP64 instances hold f at its FP64 size; unknown precisions are rejected."""
    base = dict(nx=64, qx_half=4, qy=4, qz=4, kn=0.1, eta0=0.1)
    b64 = F.workspace_bytes([F.Params(**base, precision="fp64")])
    b32 = F.workspace_bytes([F.Params(**base, precision="fp32")])
    b2 = F.workspace_bytes([F.Params(**base, precision="fp32+fp64")])
    assert b32 < b64 < b2
    c = F.Params(**base).to_c()
    c.precision = 3
    lib = F.load()
    assert lib.fdlb_workspace_bytes((F.CParams * 1)(c), 1) == 0
    assert b"precision" in lib.fdlb_last_error(None)
    c.precision = F.FP32_THEN_FP64
    # rejected before any device access
    assert lib.fdlb_step_noalloc((F.CParams * 1)(c), ctypes.c_void_p(256), 1 << 20, 1, None, None) == F.FDLB_EINVAL
    assert b"two-phase" in lib.fdlb_last_error(None)


@pytest.mark.parametrize("Q", [1, 2, 4, 6, 8, 12, 16])
def test_library_half_range_rule_matches_oracle(F, Q):
    x, w = F.quadrature("half", Q)
    r = qd.half_range_rule(Q)
    np.testing.assert_allclose(x, r.nodes, rtol=2e-15, atol=1e-14)
    np.testing.assert_allclose(w, r.weights, rtol=5e-14, atol=1e-17)


@pytest.mark.parametrize("Q", [32, 64, 100])
def test_library_half_range_rule_high_orders(F, Q):
    """The library's rules (Stieltjes on a discretised weight, compensated sums) at the orders of
    Sec. IV's large-Kn runs, against the oracle's (decimal moments): nodes to ~1e-14 absolute,
    weights to 3e-13 relative down to the smallest (~1e-107 at order 100)."""
    x, w = F.quadrature("half", Q)
    r = qd.half_range_rule(Q)
    np.testing.assert_allclose(x, r.nodes, rtol=0, atol=2e-14)
    np.testing.assert_allclose(w, r.weights, rtol=3e-13, atol=0)
    with pytest.raises(F.FdlbError):
        F.quadrature("half", 101)


@pytest.mark.parametrize("Q", [100, 200])
def test_library_full_range_rule_high_orders(F, Q):
    """The full-range orders of App. A's comparison (up to 200): nodes to 1e-14 absolute, weights
    to 1e-13 relative down to the smallest (~1e-163 at order 200)."""
    x, w = F.quadrature("full", Q)
    r = qd.full_range_rule(Q)
    np.testing.assert_allclose(x, r.nodes, rtol=0, atol=1e-14)
    np.testing.assert_allclose(w, r.weights, rtol=1e-13, atol=0)


@pytest.mark.parametrize("Q", [2, 3, 4, 6, 8, 10, 12, 16])
def test_library_full_range_rule_matches_oracle(F, Q):
    x, w = F.quadrature("full", Q)
    r = qd.full_range_rule(Q)
    np.testing.assert_allclose(x, r.nodes, atol=1e-14)
    np.testing.assert_allclose(w, r.weights, rtol=1e-14)
