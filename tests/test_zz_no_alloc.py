"""fdlb_step_noalloc: stepping for callers that cannot allocate device memory (for example
code running inside a framework that owns every device allocation, or a loop that must not
trigger the allocator).  Its scratch is a static device array inside the library; this
test checks, through the C ABI, that two calls in a row give the same state and moments as
the ordinary context path, within the FP64 parity tolerance of the other GPU tests.
Collected last on purpose (file name), so a stop-at-first-failure run has run all others."""
import numpy as np
import pytest

from gpu_common import compare, lib, oracle_for

pytestmark = pytest.mark.gpu


def test_step_noalloc_matches_context_path_twice():
    import torch
    F = lib()
    p = F.Params(nx=45, qx_half=6, qy=6, qz=0, kn=0.1, eta0=0.2, U_left=-0.42, U_right=0.42, grid="tanh")
    ref = F.Solver([p])
    state0 = ref.get_state(0)
    f0 = np.frombuffer(state0, dtype=np.float64, offset=24)
    f_dev = torch.tensor(f0, dtype=torch.float64, device="cuda")
    mom = torch.zeros(8 * p.nx, dtype=torch.float64, device="cuda")
    for call in range(2):
        F.step_noalloc(p, f_dev, 40, mom)
        ref.step(40)
        M = ref.moments(0)
        got = mom.cpu().numpy().reshape(8, p.nx)
        for j, k in enumerate(F.MOMENT_ROWS):
            scale = np.maximum(np.abs(M[k]), 1.0)
            assert np.max(np.abs(got[j] - M[k]) / scale) <= 1e-12, (call, k)
        fr = np.frombuffer(ref.get_state(0), dtype=np.float64, offset=24)
        assert np.max(np.abs(f_dev.cpu().numpy() - fr)) <= 1e-12 * np.max(np.abs(fr)), call
    # and both against the oracle after the 80 steps of the two calls
    o = oracle_for(p)
    o.step(80)
    got = mom.cpu().numpy().reshape(8, p.nx)
    compare({k: got[j] for j, k in enumerate(F.MOMENT_ROWS)}, o.moments(), 1e-12, "step_noalloc vs oracle")


def test_step_noalloc_rejects_oversize_and_bad_buffer():
    """The library's own checks, called through the C ABI directly (the binding's checks
    would stop these buffers before the library sees them)."""
    import ctypes
    import torch
    F = lib()
    L = F.load()
    f_dev = torch.zeros(16, dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    big = F.Params(nx=4096, qx_half=16, qy=8, qz=8, kn=0.1, eta0=0.1).to_c()
    rc = L.fdlb_step_noalloc(ctypes.byref(big), ctypes.c_void_p(f_dev.data_ptr()), 16 * 8, 1, None, st)
    assert rc == F.FDLB_ENOMEM and "static maximum" in L.fdlb_last_error(None).decode()
    p = F.Params(nx=16, qx_half=4, qy=4, qz=0, kn=0.1, eta0=0.1).to_c()
    rc = L.fdlb_step_noalloc(ctypes.byref(p), ctypes.c_void_p(f_dev.data_ptr()), 16 * 8, 1, None, st)
    assert rc == F.FDLB_EINVAL and "f_bytes" in L.fdlb_last_error(None).decode()
