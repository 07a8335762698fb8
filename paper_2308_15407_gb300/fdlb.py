"""ctypes binding of the C ABI in include/fdlb.h (argument marshalling only).

Every step of the solver runs in the CUDA kernels of libfdlb.so.  PyTorch is used
only to allocate the device workspace and to name the CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field, fields

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfdlb.so")

FDLB_OK, FDLB_EINVAL, FDLB_ENOMEM, FDLB_ECUDA, FDLB_ENONFINITE, FDLB_EUNPHYSICAL, FDLB_ETIMEOUT, FDLB_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
FOURIER, COUETTE, POISEUILLE = 0, 1, 2
GRID_UNIFORM, GRID_TANH = 0, 1
FP64, FP32_STORAGE, FP32_THEN_FP64 = 0, 1, 2
CHI_SET, CHI_RET_FM = 0, 1
XQ_HALF, XQ_FULL = 0, 1
PRECISIONS = {"fp64": FP64, "fp32": FP32_STORAGE, "fp32+fp64": FP32_THEN_FP64}
SCHED_AUTO, SCHED_TILED, SCHED_RESIDENT, SCHED_MIXED = 0, 1, 2, 3
SCHEDULES = {"auto": SCHED_AUTO, "tiled": SCHED_TILED, "resident": SCHED_RESIDENT, "mixed": SCHED_MIXED}
ACTIVE, CONVERGED, FAILED_NONFINITE, FAILED_UNPHYSICAL, STAGNATED, FAILED_COPY = 0, 1, 2, 3, 4, 5
MOMENT_ROWS = ("n", "ux", "uy", "T", "qx", "qy", "Pxx", "Pxy")


class CParams(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("flow", C.c_int32), ("nx", C.c_int32), ("grid", C.c_int32),
                ("qx_half", C.c_int32), ("qy", C.c_int32), ("qz", C.c_int32), ("precision", C.c_int32),
                ("j1_shear", C.c_int32), ("chi_model", C.c_int32), ("x_quadrature", C.c_int32),
                ("stretch", C.c_double), ("kn", C.c_double),
                ("eta0", C.c_double), ("T_left", C.c_double), ("T_right", C.c_double), ("U_left", C.c_double),
                ("U_right", C.c_double), ("accel_y", C.c_double), ("cfl", C.c_double), ("dt", C.c_double),
                ("T_init", C.c_double)]


@dataclass
class Params:
    """One channel problem (field meanings as in ``fdlb_params``)."""
    nx: int
    qx_half: int
    qy: int
    qz: int
    kn: float
    eta0: float
    T_left: float = 1.0
    T_right: float = 1.0
    U_left: float = 0.0
    U_right: float = 0.0
    accel_y: float = 0.0
    grid: str = "uniform"
    stretch: float = 1.5
    cfl: float = 0.5
    dt: float = 0.0
    j1_shear: bool = False
    flow: int = FOURIER
    T_init: float = 0.0
    precision: str = "fp64"
    chi_model: str = "set"
    x_quadrature: str = "half"      # "half" (Sec. III A 2) or "full" (order 2 qx_half, App. A)

    def to_c(self) -> CParams:
        p = CParams()
        p.struct_size = C.sizeof(CParams)
        p.flow = int(self.flow)
        p.nx = int(self.nx)
        p.grid = {"uniform": GRID_UNIFORM, "tanh": GRID_TANH}[self.grid]
        p.qx_half, p.qy, p.qz = int(self.qx_half), int(self.qy), int(self.qz)
        p.precision = PRECISIONS[self.precision]
        p.j1_shear = int(bool(self.j1_shear))
        p.chi_model = {"set": CHI_SET, "ret-fm": CHI_RET_FM}[self.chi_model]
        p.x_quadrature = {"half": XQ_HALF, "full": XQ_FULL}[self.x_quadrature]
        p.stretch, p.kn, p.eta0 = float(self.stretch), float(self.kn), float(self.eta0)
        p.T_left, p.T_right, p.U_left, p.U_right = float(self.T_left), float(self.T_right), float(self.U_left), float(self.U_right)
        p.accel_y, p.cfl, p.dt, p.T_init = float(self.accel_y), float(self.cfl), float(self.dt), float(self.T_init)
        return p


_lib = None


def load() -> C.CDLL:
    """Load libfdlb.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2308_15407_gb300.build`")
    lib = C.CDLL(LIB_PATH)
    P = C.POINTER(CParams)
    vp, dp, ip, lp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64)
    sig = {
        "fdlb_abi_version": (C.c_int32, []),
        "fdlb_last_error": (C.c_char_p, [vp]),
        "fdlb_workspace_bytes": (C.c_size_t, [P, C.c_int32]),
        "fdlb_create": (C.c_int, [C.POINTER(vp), P, C.c_int32, vp, C.c_size_t, vp]),
        "fdlb_destroy": (None, [vp]),
        "fdlb_info": (C.c_int, [vp, C.c_int32, ip, ip, dp]),
        "fdlb_layout": (C.c_int, [vp, C.c_int32, ip, ip, ip]),
        "fdlb_step": (C.c_int, [vp, C.c_int64, C.c_double]),
        "fdlb_run": (C.c_int, [vp, C.c_double, C.c_int64, C.c_int64, C.c_double]),
        "fdlb_moments": (C.c_int, [vp, C.c_int32, dp]),
        "fdlb_status": (C.c_int, [vp, dp, ip, lp]),
        "fdlb_residual": (C.c_int, [vp, dp]),
        "fdlb_precision": (C.c_int, [vp, ip, lp]),
        "fdlb_set_schedule": (C.c_int, [vp, C.c_int32]),
        "fdlb_get_schedule": (C.c_int, [vp, ip, ip]),
        "fdlb_get_schedule_mix": (C.c_int, [vp, ip, ip]),
        "fdlb_set_profiles": (C.c_int, [vp, C.c_int32, dp, dp, dp]),
        "fdlb_state_bytes": (C.c_size_t, [vp, C.c_int32]),
        "fdlb_get_state": (C.c_int, [vp, C.c_int32, vp, C.c_size_t]),
        "fdlb_set_state": (C.c_int, [vp, C.c_int32, vp, C.c_size_t]),
        "fdlb_quadrature": (C.c_int, [C.c_int32, C.c_int32, dp, dp]),
        "fdlb_step_noalloc": (C.c_int, [P, vp, C.c_size_t, C.c_int64, dp, vp]),
        "fdlb_mlp_param_count": (C.c_int32, []),
        "fdlb_mlp_workspace_bytes": (C.c_size_t, [C.c_int32]),
        "fdlb_mlp_last_error": (C.c_char_p, [vp]),
        "fdlb_mlp_create": (C.c_int, [C.POINTER(vp), vp, C.c_size_t, C.c_int32, C.c_uint64, vp]),
        "fdlb_mlp_destroy": (None, [vp]),
        "fdlb_mlp_get_params": (C.c_int, [vp, C.POINTER(C.c_float)]),
        "fdlb_mlp_set_params": (C.c_int, [vp, C.POINTER(C.c_float)]),
        "fdlb_mlp_predict": (C.c_int, [vp, vp, C.c_int32, vp]),
        "fdlb_mlp_train_step": (C.c_int, [vp, vp, vp, C.c_int32, C.c_float, vp, dp]),
        "fdlb_profile": (C.c_int, [vp, C.c_int32]),
        "fdlb_profile_read": (C.c_int, [vp, C.c_int32, dp, lp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class FdlbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fdlb error {code}: {msg}")
        self.code = code


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def quadrature(kind: str, q: int):
    """The library's own Gauss rule: kind 'half' (Sec. III A 2) or 'full' (App. A)."""
    lib = load()
    x = np.zeros(q)
    w = np.zeros(q)
    rc = lib.fdlb_quadrature({"half": 0, "full": 1}[kind], q, _dptr(x), _dptr(w))
    if rc != FDLB_OK:
        raise FdlbError(rc, lib.fdlb_last_error(None).decode())
    return x, w


def noalloc_f_elements(params: Params) -> int:
    """Values of f of one instance in the layout of include/fdlb.h: K x ceil(nx/32)*32."""
    tc = params.qy * params.qz if params.qz else (2 * params.qy if params.qy else 2)
    return 2 * params.qx_half * tc * ((params.nx + 31) // 32 * 32)


def step_noalloc(params: Params, f_dev, nsteps: int, moments_dev=None, stream=None) -> None:
    """fdlb_step_noalloc: advance one instance whose f lives in the caller's device tensor
    f_dev (in place), with no device allocation by the library; moments_dev (float64 device
    tensor of at least 8*nx values on f_dev's device) receives the moment rows.

    The buffers are checked here before the library sees their addresses: f_dev must be a
    contiguous tensor of float64 (precision "fp64") or float32 (precision "fp32") holding
    exactly the instance's f; moments_dev must be contiguous float64 with numel >= 8*nx on
    the same CUDA device.  A violation raises ValueError and launches nothing."""
    import torch
    want = {"fp64": torch.float64, "fp32": torch.float32}.get(params.precision)
    if want is None:
        raise ValueError(f"step_noalloc: precision {params.precision!r} is not supported (fp64 or fp32)")
    if f_dev.dtype != want:
        raise ValueError(f"step_noalloc: f_dev is {f_dev.dtype}, precision {params.precision!r} needs {want}")
    if not f_dev.is_contiguous():
        raise ValueError("step_noalloc: f_dev must be contiguous")
    nf = noalloc_f_elements(params)
    if f_dev.numel() != nf:
        raise ValueError(f"step_noalloc: f_dev has {f_dev.numel()} values, this instance's f has {nf}")
    if moments_dev is not None:
        if moments_dev.dtype != torch.float64:
            raise ValueError(f"step_noalloc: moments_dev is {moments_dev.dtype}, needs torch.float64")
        if not moments_dev.is_contiguous():
            raise ValueError("step_noalloc: moments_dev must be contiguous")
        if moments_dev.numel() < 8 * params.nx:
            raise ValueError(f"step_noalloc: moments_dev has {moments_dev.numel()} values, needs {8 * params.nx}")
        if moments_dev.device != f_dev.device:
            raise ValueError(f"step_noalloc: moments_dev is on {moments_dev.device}, f_dev on {f_dev.device}")
    if f_dev.device.type != "cuda":
        raise ValueError(f"step_noalloc: f_dev must be a CUDA tensor, not on {f_dev.device}")
    lib = load()
    c = params.to_c()
    st = stream if stream is not None else torch.cuda.current_stream(f_dev.device)
    mp = C.cast(C.c_void_p(moments_dev.data_ptr()), C.POINTER(C.c_double)) if moments_dev is not None else None
    with torch.cuda.device(f_dev.device):
        rc = lib.fdlb_step_noalloc(C.byref(c), C.c_void_p(f_dev.data_ptr()), f_dev.numel() * f_dev.element_size(),
                                   int(nsteps), mp, C.c_void_p(st.cuda_stream))
    if rc != FDLB_OK:
        raise FdlbError(rc, lib.fdlb_last_error(None).decode())


def workspace_bytes(params) -> int:
    lib = load()
    arr = (CParams * len(params))(*[p.to_c() for p in params])
    n = lib.fdlb_workspace_bytes(arr, len(params))
    if n == 0:
        raise FdlbError(FDLB_EINVAL, lib.fdlb_last_error(None).decode())
    return n


class Solver:
    """A batch of channel problems living in one device workspace."""

    def __init__(self, params, device="cuda", stream=None):
        import torch
        self.lib = load()
        if isinstance(params, Params):
            params = [params]
        self.params = list(params)
        self.count = len(self.params)
        arr = (CParams * self.count)(*[p.to_c() for p in self.params])
        nbytes = self.lib.fdlb_workspace_bytes(arr, self.count)
        if nbytes == 0:
            raise FdlbError(FDLB_EINVAL, self.lib.fdlb_last_error(None).decode())
        self.device = torch.device(device)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        ptr = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        if self.stream != torch.cuda.current_stream(self.device):
            # the library's work runs on self.stream: keep the caching allocator from reusing
            # the workspace before that work has finished
            self.ws.record_stream(self.stream)
        self.ctx = C.c_void_p()
        rc = self.lib.fdlb_create(C.byref(self.ctx), arr, self.count, C.c_void_p(ptr), nbytes,
                                  C.c_void_p(self.stream.cuda_stream))
        if rc != FDLB_OK:
            raise FdlbError(rc, self.lib.fdlb_last_error(None).decode())
        self.nx, self.nvel, self.dt = [], [], []
        for i in range(self.count):
            nx, nv, dt = C.c_int32(), C.c_int32(), C.c_double()
            self._check(self.lib.fdlb_info(self.ctx, i, C.byref(nx), C.byref(nv), C.byref(dt)))
            self.nx.append(nx.value)
            self.nvel.append(nv.value)
            self.dt.append(dt.value)

    def _check(self, rc):
        if rc < 0:
            raise FdlbError(rc, self.lib.fdlb_last_error(self.ctx).decode())
        return rc

    def close(self):
        if self.ctx:
            self.lib.fdlb_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps: int = 1, freeze_tol: float = 0.0):
        self._check(self.lib.fdlb_step(self.ctx, int(nsteps), float(freeze_tol)))
        return self

    def run(self, tol: float, max_steps: int, check_every: int = 100, timeout_s: float = 3600.0) -> int:
        return self._check(self.lib.fdlb_run(self.ctx, float(tol), int(max_steps), int(check_every), float(timeout_s)))

    def moments(self, inst: int = 0) -> dict:
        out = np.zeros((8, self.nx[inst]))
        self._check(self.lib.fdlb_moments(self.ctx, inst, _dptr(out)))
        return {k: out[j].copy() for j, k in enumerate(MOMENT_ROWS)}

    def status(self):
        r = np.zeros(self.count)
        s = np.zeros(self.count, dtype=np.int32)
        st = np.zeros(self.count, dtype=np.int64)
        self._check(self.lib.fdlb_status(self.ctx, _dptr(r), s.ctypes.data_as(C.POINTER(C.c_int32)),
                                         st.ctypes.data_as(C.POINTER(C.c_int64))))
        return r, s, st

    def residual(self) -> np.ndarray:
        """Per-instance residual of the last step (the first array of ``status``)."""
        r = np.zeros(self.count)
        self._check(self.lib.fdlb_residual(self.ctx, _dptr(r)))
        return r

    def layout(self, inst: int = 0):
        """(velocities per update block, update blocks per 32-node tile, tiles) of instance inst."""
        ch, g, t = C.c_int32(), C.c_int32(), C.c_int32()
        self._check(self.lib.fdlb_layout(self.ctx, inst, C.byref(ch), C.byref(g), C.byref(t)))
        return ch.value, g.value, t.value

    def set_schedule(self, schedule: str):
        """'auto' (time every available schedule on the first long step call), 'tiled',
        'resident' (one thread-block cluster per instance) or 'mixed' (instances that fit keep f
        in shared memory, the others tiled)."""
        self._check(self.lib.fdlb_set_schedule(self.ctx, SCHEDULES[schedule]))

    def schedule(self):
        """(schedule in use: 'auto' while not chosen, 'tiled' or 'resident'; CTAs per cluster)."""
        sc, cs = C.c_int32(), C.c_int32()
        self._check(self.lib.fdlb_get_schedule(self.ctx, C.byref(sc), C.byref(cs)))
        return {v: k for k, v in SCHEDULES.items()}[sc.value], cs.value

    def schedule_mix(self) -> np.ndarray:
        """Per instance 1 if FDLB_SCHED_MIXED keeps it in shared memory, else 0."""
        out = np.zeros(self.count, dtype=np.int32)
        n = C.c_int32()
        self._check(self.lib.fdlb_get_schedule_mix(self.ctx, out.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(n)))
        return out

    def precision_state(self):
        """(storage precision in use per instance, step of the FP32 -> FP64 switch or -1)."""
        pr = np.zeros(self.count, dtype=np.int32)
        sw = np.zeros(self.count, dtype=np.int64)
        self._check(self.lib.fdlb_precision(self.ctx, pr.ctypes.data_as(C.POINTER(C.c_int32)),
                                            sw.ctypes.data_as(C.POINTER(C.c_int64))))
        return pr, sw

    def set_profiles(self, inst: int, n, uy, T):
        n, uy, T = (np.ascontiguousarray(x, dtype=np.float64) for x in (n, uy, T))
        self._check(self.lib.fdlb_set_profiles(self.ctx, inst, _dptr(n), _dptr(uy), _dptr(T)))

    def get_state(self, inst: int = 0) -> bytes:
        nb = self.lib.fdlb_state_bytes(self.ctx, inst)
        buf = C.create_string_buffer(nb)
        self._check(self.lib.fdlb_get_state(self.ctx, inst, buf, nb))
        return buf.raw

    KERNEL_KINDS = ("moments", "nodal", "update", "resid")

    def profile(self, on: bool):
        """Start (clearing) or stop the per-kernel-class CUDA event timing."""
        self._check(self.lib.fdlb_profile(self.ctx, int(bool(on))))

    def profile_read(self) -> dict:
        """{kind: (total_ms, launches)} of the recorded launches (synchronises)."""
        out = {}
        for j, name in enumerate(self.KERNEL_KINDS):
            ms, n = C.c_double(), C.c_int64()
            self._check(self.lib.fdlb_profile_read(self.ctx, j, C.byref(ms), C.byref(n)))
            out[name] = (ms.value, n.value)
        return out

    def set_state(self, inst: int, state: bytes):
        buf = C.create_string_buffer(state, len(state))
        self._check(self.lib.fdlb_set_state(self.ctx, inst, buf, len(state)))


class MLP:
    """Warm-start network (tcgen05 BF16 kernels with FP32 accumulation) in a device workspace."""

    NIN, NOUT = 16, 3

    def __init__(self, max_points: int, seed: int = 1, device="cuda", stream=None):
        import torch
        self.lib = load()
        self.max_points = int(max_points)
        self.device = torch.device(device)
        nb = self.lib.fdlb_mlp_workspace_bytes(self.max_points)
        self.ws = torch.empty(nb + 256, dtype=torch.uint8, device=self.device)
        ptr = (self.ws.data_ptr() + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.h = C.c_void_p()
        rc = self.lib.fdlb_mlp_create(C.byref(self.h), C.c_void_p(ptr), nb, self.max_points, int(seed),
                                      C.c_void_p(self.stream.cuda_stream))
        if rc != FDLB_OK:
            raise FdlbError(rc, self.lib.fdlb_mlp_last_error(None).decode())
        self.nparam = self.lib.fdlb_mlp_param_count()

    def _check(self, rc):
        if rc < 0:
            raise FdlbError(rc, self.lib.fdlb_mlp_last_error(self.h).decode())

    def close(self):
        if self.h:
            self.lib.fdlb_mlp_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.nparam, dtype=np.float32)
        self._check(self.lib.fdlb_mlp_get_params(self.h, out.ctypes.data_as(C.POINTER(C.c_float))))
        return out

    def set_params(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        self._check(self.lib.fdlb_mlp_set_params(self.h, theta.ctypes.data_as(C.POINTER(C.c_float))))

    def predict(self, x):
        """x: float32 device tensor [P, 16] -> float32 device tensor [P, 3]."""
        import torch
        x = x.contiguous()
        y = torch.empty((x.shape[0], self.NOUT), dtype=torch.float32, device=x.device)
        self._check(self.lib.fdlb_mlp_predict(self.h, C.c_void_p(x.data_ptr()), x.shape[0], C.c_void_p(y.data_ptr())))
        return y

    def train_step(self, x, y, lr: float, want_grad: bool = False):
        """One Adam step (lr = 0: gradient only).  Returns (loss before the step, gradient or None)."""
        import torch
        x = x.contiguous()
        y = y.contiguous()
        g = torch.empty(self.nparam, dtype=torch.float32, device=x.device) if want_grad else None
        loss = C.c_double()
        self._check(self.lib.fdlb_mlp_train_step(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), x.shape[0],
                                                 float(lr), C.c_void_p(g.data_ptr()) if g is not None else None,
                                                 C.byref(loss)))
        return loss.value, g
