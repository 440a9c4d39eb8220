"""GB300-native GLM-MHD hot path: Python binding of the C ABI in include/mhd.h.

The binding only marshals arguments: every step of the method runs in the
CUDA kernels of ``libmhd_gb300.so`` (built in-tree by ``build.py``).  PyTorch
provides device memory (the workspace and user tensors) and the CUDA stream.
If the library is missing, every call raises: there is no CPU fallback.

Functions with the ABI's names (``mhd_create``, ``mhd_set_state``,
``mhd_step``, ``mhd_dt``, ``mhd_adjoint_step``, ``mhd_destroy`` ...) take the
same arguments as the C functions (device pointers as torch tensors); the
``MHD`` class wraps one context and owns its workspace tensor.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import inputs  # noqa: F401  (seeded input generators, no method arithmetic)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmhd_gb300.so")

MHD_OK, MHD_ERR_INVALID, MHD_ERR_NOMEM, MHD_ERR_CUDA = 0, -1, -2, -3
MHD_ERR_NONFINITE, MHD_ERR_TIMEOUT, MHD_ERR_STATE = -4, -5, -6
MHD_LIM_FLAT, MHD_LIM_MINMOD, MHD_LIM_MC, MHD_LIM_WENOZ = 0, 1, 2, 3
MHD_BC_PERIODIC, MHD_BC_OUTFLOW, MHD_BC_HALO = 0, 1, 2
MHD_FP64, MHD_FP32 = 0, 1
MHD_HOST, MHD_DEVICE = 0, 1
MHD_CONS, MHD_PRIM = 0, 1
MHD_FLAG_ADJOINT = 1
MHD_DIVB_GLM, MHD_DIVB_CT = 0, 1

EXPORTED = ["mhd_config_default", "mhd_workspace_bytes", "mhd_create", "mhd_set_stream",
            "mhd_set_state", "mhd_get_state", "mhd_dt", "mhd_step", "mhd_step_host",
            "mhd_step_n", "mhd_step_info", "mhd_step_record",
            "mhd_counters", "mhd_conserved_sums", "mhd_flux_batch", "mhd_adjoint_step",
            "mhd_adjoint_step_stage1", "mhd_get_stage1",
            "mhd_profile_enable", "mhd_profile_read", "mhd_conserved_sums_noalloc",
            "mhd_last_error", "mhd_destroy", "mhd_set_face_field", "mhd_get_face_field",
            "mhd_divb_max", "mhd_halo_bytes", "mhd_halo_pack", "mhd_lambda_max_into",
            "mhd_step_begin", "mhd_step_stage",
            "mhd_ensemble_workspace_bytes", "mhd_ensemble_create", "mhd_ensemble_set_state",
            "mhd_ensemble_get_state", "mhd_ensemble_step", "mhd_ensemble_info",
            "mhd_ensemble_autotune", "mhd_ensemble_set_tiles", "mhd_ensemble_last_error",
            "mhd_ensemble_destroy", "mhd_fp64_fma_rate", "mhd_plan_z_chunks"]


class MHDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"MHD error {code}: {msg}")
        self.code = code


class mhd_config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("xmin", ctypes.c_double * 3),
                ("xmax", ctypes.c_double * 3), ("gamma", ctypes.c_double),
                ("cfl", ctypes.c_double), ("glm_alpha", ctypes.c_double),
                ("rho_floor", ctypes.c_double), ("p_floor", ctypes.c_double),
                ("t_end", ctypes.c_double), ("limiter", ctypes.c_int),
                ("bc", ctypes.c_int * 6), ("precision", ctypes.c_int), ("flags", ctypes.c_int),
                ("rk_order", ctypes.c_int), ("divb", ctypes.c_int),
                ("dx", ctypes.c_double * 3)]


_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"CUDA library {LIB_PATH} is missing: run paper_2510_24175_gb300/build.py "
                "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        cfgp = ctypes.POINTER(mhd_config)
        dp = ctypes.POINTER(ctypes.c_double)
        L.mhd_config_default.argtypes = [cfgp]
        L.mhd_workspace_bytes.argtypes = [cfgp, ctypes.POINTER(ctypes.c_size_t)]
        L.mhd_create.argtypes = [cfgp, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
        L.mhd_set_stream.argtypes = [vp, vp]
        L.mhd_set_state.argtypes = [vp, vp, i, i]
        L.mhd_get_state.argtypes = [vp, vp, i, i]
        L.mhd_set_face_field.argtypes = [vp, vp, i]
        L.mhd_get_face_field.argtypes = [vp, vp, i]
        L.mhd_divb_max.argtypes = [vp, dp]
        L.mhd_dt.argtypes = [vp, dp, dp]
        L.mhd_step.argtypes = [vp, d, d]
        L.mhd_step_host.argtypes = [vp, vp, vp, d, d]
        L.mhd_step_n.argtypes = [vp, i]
        L.mhd_step_info.argtypes = [vp, dp]
        L.mhd_step_record.argtypes = [vp, vp]
        L.mhd_counters.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
        L.mhd_conserved_sums.argtypes = [vp, dp]
        L.mhd_flux_batch.argtypes = [vp, vp, vp, ctypes.c_longlong, i, d, d, i, vp]
        L.mhd_fp64_fma_rate.argtypes = [vp, ctypes.c_uint, ctypes.POINTER(ctypes.c_double)]
        L.mhd_plan_z_chunks.argtypes = [ctypes.POINTER(ctypes.c_int), i, i, i,
                                        ctypes.POINTER(ctypes.c_int), dp]
        L.mhd_adjoint_step.argtypes = [vp, vp, vp, vp, d, d]
        L.mhd_adjoint_step_stage1.argtypes = [vp, vp, vp, vp, vp, d, d]
        L.mhd_get_stage1.argtypes = [vp, vp, i]
        L.mhd_profile_enable.argtypes = [vp, i]
        L.mhd_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), dp]
        L.mhd_conserved_sums_noalloc.argtypes = [cfgp, vp, dp, vp]
        L.mhd_last_error.argtypes = [vp]
        L.mhd_last_error.restype = ctypes.c_char_p
        L.mhd_ensemble_workspace_bytes.argtypes = [cfgp, i, ctypes.POINTER(ctypes.c_size_t)]
        L.mhd_ensemble_create.argtypes = [cfgp, i, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
        L.mhd_ensemble_set_state.argtypes = [vp, i, vp, i, i]
        L.mhd_ensemble_get_state.argtypes = [vp, i, vp, i, i]
        L.mhd_ensemble_step.argtypes = [vp, i]
        L.mhd_ensemble_info.argtypes = [vp, i, dp]
        L.mhd_ensemble_autotune.argtypes = [vp, i]
        L.mhd_ensemble_set_tiles.argtypes = [vp, i, i, i]
        L.mhd_ensemble_last_error.argtypes = [vp]
        L.mhd_ensemble_last_error.restype = ctypes.c_char_p
        L.mhd_ensemble_destroy.argtypes = [vp]
        L.mhd_destroy.argtypes = [vp]
        L.mhd_halo_bytes.argtypes = [vp, i, ctypes.POINTER(ctypes.c_size_t)]
        L.mhd_halo_pack.argtypes = [vp, i, vp]
        L.mhd_lambda_max_into.argtypes = [vp, vp]
        L.mhd_step_begin.argtypes = [vp, d, d, vp]
        L.mhd_step_stage.argtypes = [vp, ctypes.POINTER(vp)]
        for name in EXPORTED:
            if not name.endswith("last_error"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int, ctx=None, what: str = ""):
    if rc != MHD_OK:
        # no context: the calling thread's last context-free message
        msg = lib().mhd_last_error(ctx if ctx else None).decode()
        raise MHDError(rc, f"{what}: {msg}")


def _torch():
    import torch
    return torch


def _stream_ptr():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------ ABI functions --
def mhd_config_default() -> mhd_config:
    c = mhd_config()
    _check(lib().mhd_config_default(ctypes.byref(c)), what="mhd_config_default")
    return c


def mhd_workspace_bytes(cfg: mhd_config) -> int:
    b = ctypes.c_size_t()
    _check(lib().mhd_workspace_bytes(ctypes.byref(cfg), ctypes.byref(b)),
           what="mhd_workspace_bytes")
    return b.value


def mhd_create(cfg: mhd_config, workspace, stream=None) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    s = stream if stream is not None else _stream_ptr()
    _check(lib().mhd_create(ctypes.byref(cfg), _ptr(workspace), workspace.numel(), s,
                            ctypes.byref(ctx)), what="mhd_create")
    return ctx


def mhd_set_state(ctx, U, where=MHD_DEVICE, kind=MHD_CONS):
    p = _ptr(U) if where == MHD_DEVICE else U.ctypes.data_as(ctypes.c_void_p)
    _check(lib().mhd_set_state(ctx, p, where, kind), ctx, "mhd_set_state")


def mhd_get_state(ctx, U, where=MHD_DEVICE, kind=MHD_CONS):
    p = _ptr(U) if where == MHD_DEVICE else U.ctypes.data_as(ctypes.c_void_p)
    _check(lib().mhd_get_state(ctx, p, where, kind), ctx, "mhd_get_state")


def mhd_set_face_field(ctx, b, where=MHD_DEVICE):
    p = _ptr(b) if where == MHD_DEVICE else b.ctypes.data_as(ctypes.c_void_p)
    _check(lib().mhd_set_face_field(ctx, p, where), ctx, "mhd_set_face_field")


def mhd_get_face_field(ctx, b, where=MHD_DEVICE):
    p = _ptr(b) if where == MHD_DEVICE else b.ctypes.data_as(ctypes.c_void_p)
    _check(lib().mhd_get_face_field(ctx, p, where), ctx, "mhd_get_face_field")


def mhd_divb_max(ctx) -> float:
    out = ctypes.c_double()
    _check(lib().mhd_divb_max(ctx, ctypes.byref(out)), ctx, "mhd_divb_max")
    return out.value


def mhd_dt(ctx):
    dt, ch = ctypes.c_double(), ctypes.c_double()
    _check(lib().mhd_dt(ctx, ctypes.byref(dt), ctypes.byref(ch)), ctx, "mhd_dt")
    return dt.value, ch.value


def mhd_step(ctx, dt: float = 0.0, ch: float = 0.0):
    _check(lib().mhd_step(ctx, float(dt), float(ch)), ctx, "mhd_step")


def mhd_step_record(ctx, out):
    """(t, dt, c_h, steps) of the last step into ``out`` (4 float64 values of
    a CUDA tensor), enqueued without synchronising."""
    _check(lib().mhd_step_record(ctx, _ptr(out)), ctx, "mhd_step_record")


def mhd_halo_bytes(ctx, face: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().mhd_halo_bytes(ctx, int(face), ctypes.byref(b)), ctx, "mhd_halo_bytes")
    return b.value


def mhd_halo_pack(ctx, face: int, dst):
    """The g boundary layers next to ``face`` of the next stage's input into
    ``dst`` (a CUDA tensor of mhd_halo_bytes bytes)."""
    _check(lib().mhd_halo_pack(ctx, int(face), _ptr(dst)), ctx, "mhd_halo_pack")


def mhd_lambda_max_into(ctx, bits):
    """Raises ``bits`` (a one-element int64 CUDA tensor) to the context's
    maximum wave speed, as FP64 bits."""
    _check(lib().mhd_lambda_max_into(ctx, _ptr(bits)), ctx, "mhd_lambda_max_into")


def mhd_step_begin(ctx, dt: float = 0.0, ch: float = 0.0, lam_bits=None):
    p = _ptr(lam_bits) if lam_bits is not None else None
    _check(lib().mhd_step_begin(ctx, float(dt), float(ch), p), ctx, "mhd_step_begin")


def mhd_step_stage(ctx, halo=None):
    """halo: six CUDA tensors or None (faces without halo buffers)."""
    arr = None
    if halo is not None:
        arr = (ctypes.c_void_p * 6)(*[(t.data_ptr() if t is not None else None) for t in halo])
    _check(lib().mhd_step_stage(ctx, arr), ctx, "mhd_step_stage")


def mhd_step_n(ctx, nsteps: int):
    _check(lib().mhd_step_n(ctx, int(nsteps)), ctx, "mhd_step_n")


def mhd_step_host(ctx, U_in, U_out, dt: float = 0.0, ch: float = 0.0):
    """U_in, U_out: float64 numpy arrays (9, nz, ny, nx) in host memory
    (page-locked for the copy overlap); U_out may be U_in."""
    _check(lib().mhd_step_host(ctx, U_in.ctypes.data_as(ctypes.c_void_p),
                               U_out.ctypes.data_as(ctypes.c_void_p), float(dt), float(ch)),
           ctx, "mhd_step_host")


def mhd_adjoint_step(ctx, U_n, lam_np1, lam_n, dt: float, ch: float):
    _check(lib().mhd_adjoint_step(ctx, _ptr(U_n), _ptr(lam_np1), _ptr(lam_n), float(dt),
                                  float(ch)), ctx, "mhd_adjoint_step")


def mhd_adjoint_step_stage1(ctx, U_n, U1, lam_np1, lam_n, dt: float, ch: float):
    _check(lib().mhd_adjoint_step_stage1(ctx, _ptr(U_n), _ptr(U1), _ptr(lam_np1), _ptr(lam_n),
                                         float(dt), float(ch)), ctx, "mhd_adjoint_step_stage1")


def mhd_get_stage1(ctx, U1, where: int):
    p = _ptr(U1) if where == MHD_DEVICE else U1.ctypes.data_as(ctypes.c_void_p)
    _check(lib().mhd_get_stage1(ctx, p, int(where)), ctx, "mhd_get_stage1")


def mhd_destroy(ctx):
    _check(lib().mhd_destroy(ctx), what="mhd_destroy")


def mhd_conserved_sums_noalloc(cfg: mhd_config, U) -> np.ndarray:
    """Conservation sums of a caller-held CUDA state tensor (float64 or
    float32 to match cfg.precision) without a context or workspace; the
    library's fixed internal scratch is used and nothing is allocated.  The
    current stream must not be capturing (the call synchronises it)."""
    torch = _torch()
    want = torch.float64 if cfg.precision == MHD_FP64 else torch.float32
    ncell = int(cfg.n[0]) * int(cfg.n[1]) * int(cfg.n[2])
    assert U.is_cuda and U.is_contiguous(), "U must be a contiguous CUDA tensor"
    assert U.dtype == want, f"U is {U.dtype}, the config's precision needs {want}"
    assert U.numel() >= 9 * ncell, f"U holds {U.numel()} values, the grid needs {9 * ncell}"
    out = (ctypes.c_double * 8)()
    _check(lib().mhd_conserved_sums_noalloc(ctypes.byref(cfg), _ptr(U), out, _stream_ptr()),
           what="mhd_conserved_sums_noalloc")
    return np.array(out[:])


def mhd_flux_batch(VL, VR, F, direction: int, ch: float, gamma: float):
    """GLM + HLLD fluxes of face pairs; VL, VR, F: CUDA tensors (9, nface),
    float64 or float32."""
    torch = _torch()
    prec = MHD_FP64 if VL.dtype == torch.float64 else MHD_FP32
    for t in (VL, VR, F):
        assert t.is_cuda and t.is_contiguous() and t.shape[0] == 9 and t.dtype == VL.dtype
    _check(lib().mhd_flux_batch(_ptr(VL), _ptr(VR), _ptr(F), VL.shape[1], direction, ch, gamma,
                                prec, _stream_ptr()), what="mhd_flux_batch")


def mhd_fp64_fma_rate(warp_mask: int = 0xFF) -> dict:
    """Measured FP64 fused multiply-add throughput of the current device, on
    the current stream, with the warps of warp_mask (of 8 per SM) running:
    lane-FMAs per second, per clock per SM, and the timed launch's
    milliseconds."""
    out = (ctypes.c_double * 3)()
    _check(lib().mhd_fp64_fma_rate(_stream_ptr(), warp_mask, out), what="mhd_fp64_fma_rate")
    return {"lane_fma_per_s": out[0], "lanes_per_clk_per_sm": out[1], "ms": out[2]}


def mhd_plan_z_chunks(n, ty: int, nsm: int, ctas_per_sm: int):
    """Host-only launch plan of the 3-D stage kernels (no GPU needed): the
    z-chunk depth for an n[0] x n[1] x n[2] grid of 32 x ty column tiles on
    nsm SMs with ctas_per_sm stage CTAs each, and the modelled launch
    duration in plane iterations."""
    nn = (ctypes.c_int * 3)(*[int(x) for x in n])
    tz = ctypes.c_int(0)
    span = ctypes.c_double(0.0)
    _check(lib().mhd_plan_z_chunks(nn, int(ty), int(nsm), int(ctas_per_sm), ctypes.byref(tz),
                                   ctypes.byref(span)), what="mhd_plan_z_chunks")
    return tz.value, span.value


# ----------------------------------------------------------------- wrapper --
@dataclass
class Config:
    n: tuple
    xmin: tuple = (0.0, 0.0, 0.0)
    xmax: tuple = (1.0, 1.0, 1.0)
    gamma: float = 5.0 / 3.0
    cfl: float = 0.8
    glm_alpha: float = 0.1
    rho_floor: float = 1e-12
    p_floor: float = 1e-12
    t_end: float = 0.0
    limiter: int = MHD_LIM_MC
    bc: tuple = (MHD_BC_PERIODIC,) * 6
    precision: int = MHD_FP64
    flags: int = 0
    rk_order: int = 2
    divb: int = MHD_DIVB_GLM
    dx: tuple = (0.0, 0.0, 0.0)  # > 0: the cell size as given (mhd_config.dx)

    @classmethod
    def from_problem(cls, pb, precision=None, flags: int = 0) -> "Config":
        return cls(n=tuple(pb.n), xmin=tuple(pb.xmin), xmax=tuple(pb.xmax), gamma=pb.gamma,
                   cfl=pb.cfl, glm_alpha=pb.glm_alpha, rho_floor=pb.rho_floor,
                   p_floor=pb.p_floor, t_end=pb.t_end, limiter=pb.limiter, bc=tuple(pb.bc),
                   precision=pb.precision if precision is None else precision, flags=flags,
                   rk_order=getattr(pb, "rk_order", 2), divb=getattr(pb, "divb", MHD_DIVB_GLM))

    def c(self) -> mhd_config:
        c = mhd_config()
        for d in range(3):
            c.n[d] = int(self.n[d])
            c.xmin[d] = float(self.xmin[d])
            c.xmax[d] = float(self.xmax[d])
        c.gamma, c.cfl, c.glm_alpha = self.gamma, self.cfl, self.glm_alpha
        c.rho_floor, c.p_floor, c.t_end = self.rho_floor, self.p_floor, self.t_end
        c.limiter, c.precision, c.flags = int(self.limiter), int(self.precision), int(self.flags)
        c.rk_order = int(self.rk_order)
        c.divb = int(self.divb)
        for s in range(6):
            c.bc[s] = int(self.bc[s])
        for d in range(3):
            c.dx[d] = float(self.dx[d])
        return c


class MHD:
    """One solver context on the current CUDA device and stream."""

    def __init__(self, config: Config, stream=None):
        torch = _torch()
        self.config = config
        self._c = config.c()
        nbytes = mhd_workspace_bytes(self._c)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        off = (-self.workspace.data_ptr()) % 256
        self._ws = self.workspace[off:off + nbytes]
        s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else _stream_ptr()
        self.ctx = ctypes.c_void_p()
        _check(lib().mhd_create(ctypes.byref(self._c), _ptr(self._ws), nbytes, s,
                                ctypes.byref(self.ctx)), what="mhd_create")
        nx, ny, nz = config.n
        self.shape = (9, nz, ny, nx)

    def __del__(self):
        try:
            if getattr(self, "ctx", None) and self.ctx.value:
                lib().mhd_destroy(self.ctx)
                self.ctx = None
        except Exception:
            pass

    def set_stream(self, stream):
        _check(lib().mhd_set_stream(self.ctx, ctypes.c_void_p(stream.cuda_stream)), self.ctx,
               "mhd_set_stream")

    def set_state(self, U, kind=MHD_CONS):
        """U: float64 CUDA tensor or numpy array of shape (9, nz, ny, nx)."""
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.float64)
            assert U.shape == self.shape
            mhd_set_state(self.ctx, U, MHD_HOST, kind)
        else:
            torch = _torch()
            assert U.is_cuda and U.dtype == torch.float64 and U.is_contiguous()
            assert tuple(U.shape) == self.shape
            mhd_set_state(self.ctx, U, MHD_DEVICE, kind)

    def set_face_field(self, b):
        """Constrained transport: face field b of shape (3, nz, ny, nx), float64
        (CUDA tensor or numpy array); b[d] on each cell's lower d-face."""
        shape = (3,) + self.shape[1:]
        if isinstance(b, np.ndarray):
            b = np.ascontiguousarray(b, dtype=np.float64)
            assert b.shape == shape
            mhd_set_face_field(self.ctx, b, MHD_HOST)
        else:
            torch = _torch()
            assert b.is_cuda and b.dtype == torch.float64 and b.is_contiguous()
            assert tuple(b.shape) == shape
            mhd_set_face_field(self.ctx, b, MHD_DEVICE)

    def get_face_field(self, out=None):
        """Constrained transport: the face field as a float64 CUDA tensor (or
        into ``out``; a numpy ``out`` receives a host copy)."""
        torch = _torch()
        if out is None:
            out = torch.empty((3,) + self.shape[1:], dtype=torch.float64, device="cuda")
        mhd_get_face_field(self.ctx, out, MHD_HOST if isinstance(out, np.ndarray) else MHD_DEVICE)
        return out

    def divb_max(self) -> float:
        return mhd_divb_max(self.ctx)

    def get_state(self, out=None, kind=MHD_CONS):
        """Returns the state as a float64 CUDA tensor (or fills ``out``; a
        numpy ``out`` receives a host copy)."""
        torch = _torch()
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        if isinstance(out, np.ndarray):
            mhd_get_state(self.ctx, out, MHD_HOST, kind)
        else:
            mhd_get_state(self.ctx, out, MHD_DEVICE, kind)
        return out

    def dt(self):
        return mhd_dt(self.ctx)

    def step(self, dt: float = 0.0, ch: float = 0.0):
        mhd_step(self.ctx, dt, ch)

    def step_n(self, nsteps: int):
        """nsteps CFL steps launched as one captured CUDA graph (mhd_step_n)."""
        mhd_step_n(self.ctx, nsteps)

    def step_host(self, U_in, U_out, dt: float = 0.0, ch: float = 0.0):
        """One step of a host-resident state (mhd_step_host): U_in, U_out are
        float64 numpy arrays (9, nz, ny, nx), contiguous; U_out may be U_in."""
        for a in (U_in, U_out):
            assert isinstance(a, np.ndarray) and a.dtype == np.float64
            assert a.flags["C_CONTIGUOUS"] and a.shape == self.shape
        mhd_step_host(self.ctx, U_in, U_out, dt, ch)

    def step_info(self):
        out = (ctypes.c_double * 4)()
        _check(lib().mhd_step_info(self.ctx, out), self.ctx, "mhd_step_info")
        return {"t": out[0], "dt": out[1], "ch": out[2], "steps": int(out[3])}

    def step_record(self, out):
        """Enqueues (t, dt, c_h, steps) of the last step into ``out``, a
        float64 CUDA tensor of 4 contiguous values (no synchronisation)."""
        torch = _torch()
        assert out.is_cuda and out.dtype == torch.float64 and out.is_contiguous()
        assert out.numel() >= 4
        mhd_step_record(self.ctx, out)

    # -- staged steps and halo faces (see paper_2510_24175_gb300.decomp) --
    def halo_bytes(self, face: int) -> int:
        return mhd_halo_bytes(self.ctx, face)

    def halo_buffer(self, face: int):
        """A CUDA tensor sized for face ``face``'s halo buffer, in the
        context's precision."""
        torch = _torch()
        dt = torch.float64 if self.config.precision == MHD_FP64 else torch.float32
        es = 8 if dt == torch.float64 else 4
        return torch.empty(self.halo_bytes(face) // es, dtype=dt, device="cuda")

    def halo_pack(self, face: int, dst):
        torch = _torch()
        want = torch.float64 if self.config.precision == MHD_FP64 else torch.float32
        assert dst.is_cuda and dst.is_contiguous() and dst.dtype == want
        assert dst.numel() * dst.element_size() >= self.halo_bytes(face)
        mhd_halo_pack(self.ctx, face, dst)

    def lambda_max_into(self, bits):
        torch = _torch()
        assert bits.is_cuda and bits.dtype == torch.int64 and bits.numel() >= 1
        mhd_lambda_max_into(self.ctx, bits)

    def step_begin(self, dt: float = 0.0, ch: float = 0.0, lam_bits=None):
        if lam_bits is not None:
            torch = _torch()
            assert lam_bits.is_cuda and lam_bits.dtype == torch.int64
        mhd_step_begin(self.ctx, dt, ch, lam_bits)

    def step_stage(self, halo=None):
        if halo is not None:
            torch = _torch()
            want = torch.float64 if self.config.precision == MHD_FP64 else torch.float32
            for f, t in enumerate(halo):
                if t is not None:
                    assert t.is_cuda and t.is_contiguous() and t.dtype == want
                    assert t.numel() * t.element_size() >= self.halo_bytes(f)
        mhd_step_stage(self.ctx, halo)

    def counters(self):
        """Per-stage, per-cell counts of the floor branches of cons->prim
        (mhd_counters): rho floor, p floor, and (FP32) the pressure
        recomputed in FP64; plus the device status bits."""
        out = (ctypes.c_longlong * 4)()
        _check(lib().mhd_counters(self.ctx, out), self.ctx, "mhd_counters")
        return {"rho_floor": out[0], "p_floor": out[1], "status": out[2], "p_f64": out[3]}

    def conserved_sums(self) -> np.ndarray:
        out = (ctypes.c_double * 8)()
        _check(lib().mhd_conserved_sums(self.ctx, out), self.ctx, "mhd_conserved_sums")
        return np.array(out[:])

    def profile(self, enable: bool = True):
        _check(lib().mhd_profile_enable(self.ctx, int(enable)), self.ctx, "mhd_profile_enable")

    def profile_read(self):
        """{kernel class: (launches, total ms)} since the last read."""
        cnt = (ctypes.c_longlong * 6)()
        ms = (ctypes.c_double * 6)()
        _check(lib().mhd_profile_read(self.ctx, cnt, ms), self.ctx, "mhd_profile_read")
        names = ("prep", "stage1", "stage2", "max_speed", "stage_mid", "ct")
        return {names[k]: (int(cnt[k]), float(ms[k])) for k in range(6)}

    def adjoint_step(self, U_n, lam_np1, lam_n, dt: float, ch: float):
        mhd_adjoint_step(self.ctx, U_n, lam_np1, lam_n, dt, ch)

    def get_stage1(self, out=None):
        """The last step's first Runge-Kutta stage U1 (mhd_get_stage1) as a
        float64 CUDA tensor (or into ``out``; a numpy ``out`` receives a host
        copy)."""
        torch = _torch()
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        if isinstance(out, np.ndarray):
            assert out.dtype == np.float64 and out.flags["C_CONTIGUOUS"]
            assert out.shape == self.shape
            mhd_get_stage1(self.ctx, out, MHD_HOST)
        else:
            assert out.is_cuda and out.dtype == torch.float64 and out.is_contiguous()
            assert tuple(out.shape) == self.shape
            mhd_get_stage1(self.ctx, out, MHD_DEVICE)
        return out

    def adjoint_step_stage1(self, U_n, U1, lam_np1, lam_n, dt: float, ch: float):
        """adjoint_step with the step's first stage U1 supplied (get_stage1)."""
        mhd_adjoint_step_stage1(self.ctx, U_n, U1, lam_np1, lam_n, dt, ch)

    def run(self, nsteps: int, t_end: float = 0.0):
        """Advances up to nsteps CFL steps (stopping at t_end when the config
        sets one); returns the step info."""
        for _ in range(nsteps):
            self.step()
            if t_end > 0.0:
                info = self.step_info()
                if info["t"] >= t_end:
                    break
        return self.step_info()


class Ensemble:
    """Independent 3-D FP32 boxes advanced together by one persistent,
    graph-captured launch per ``step`` call (mhd_ensemble_*)."""

    def __init__(self, configs, stream=None):
        torch = _torch()
        self.configs = list(configs)
        n = len(self.configs)
        self._c = (mhd_config * n)(*[c.c() for c in self.configs])
        nbytes = ctypes.c_size_t()
        _check(lib().mhd_ensemble_workspace_bytes(self._c, n, ctypes.byref(nbytes)),
               what="mhd_ensemble_workspace_bytes")
        self.workspace = torch.empty(nbytes.value + 256, dtype=torch.uint8, device="cuda")
        off = (-self.workspace.data_ptr()) % 256
        ws = self.workspace[off:off + nbytes.value]
        s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else _stream_ptr()
        self.ens = ctypes.c_void_p()
        _check(lib().mhd_ensemble_create(self._c, n, _ptr(ws), nbytes.value, s,
                                         ctypes.byref(self.ens)), what="mhd_ensemble_create")
        self.shapes = [(9, c.n[2], c.n[1], c.n[0]) for c in self.configs]

    def _err(self, rc, what):
        if rc != MHD_OK:
            raise MHDError(rc, f"{what}: {lib().mhd_ensemble_last_error(self.ens).decode()}")

    def __del__(self):
        try:
            if getattr(self, "ens", None) and self.ens.value:
                lib().mhd_ensemble_destroy(self.ens)
                self.ens = None
        except Exception:
            pass

    def __len__(self):
        return len(self.configs)

    def set_state(self, box: int, U, kind=MHD_CONS):
        assert U.is_cuda and U.is_contiguous() and tuple(U.shape) == self.shapes[box]
        self._err(lib().mhd_ensemble_set_state(self.ens, box, _ptr(U), MHD_DEVICE, kind),
                  "mhd_ensemble_set_state")

    def get_state(self, box: int, kind=MHD_CONS):
        torch = _torch()
        out = torch.empty(self.shapes[box], dtype=torch.float64, device="cuda")
        self._err(lib().mhd_ensemble_get_state(self.ens, box, _ptr(out), MHD_DEVICE, kind),
                  "mhd_ensemble_get_state")
        return out

    def step(self, nsteps: int = 1):
        self._err(lib().mhd_ensemble_step(self.ens, nsteps), "mhd_ensemble_step")

    def info(self, box: int):
        out = (ctypes.c_double * 7)()
        self._err(lib().mhd_ensemble_info(self.ens, box, out), "mhd_ensemble_info")
        return {"t": out[0], "dt": out[1], "ch": out[2], "steps": int(out[3]),
                "tz": int(out[4]), "graph": bool(out[5]), "ty": int(out[6])}

    def set_tiles(self, box: int, ty: int, tz: int):
        """Tile shape of one box: 32 x ty column tiles (ty = 8 or 4), z chunks
        of tz planes (mhd_ensemble_set_tiles)."""
        self._err(lib().mhd_ensemble_set_tiles(self.ens, box, int(ty), int(tz)),
                  "mhd_ensemble_set_tiles")

    def autotune(self, trial_steps: int = 1):
        """Picks each box-size class's tile height and z-chunk depth by timing;
        the boxes' states are saved before and restored after (the trial
        launches advance them)."""
        saved = [self.get_state(b) for b in range(len(self))]
        self._err(lib().mhd_ensemble_autotune(self.ens, trial_steps), "mhd_ensemble_autotune")
        for b, U in enumerate(saved):
            self.set_state(b, U)
