"""CPU FP64 oracle for the GLM-MHD RK2 step -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It wraps ``mhd_oracle.cpp`` (a plain C++
restatement of the five per-stage steps of Section 3.2 with HLLD, Section 4.2,
and GLM divergence cleaning, Section 4.2) through ctypes.  It shares no code
with the CUDA library and never imports it.

All state arrays are interior-only SoA float64 arrays of shape (9, nz, ny, nx),
conservative ordering (rho, mx, my, mz, Bx, By, Bz, E, psi) or primitive
ordering (rho, vx, vy, vz, Bx, By, Bz, p, psi).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhd_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libmhd_oracle.so")

LIM_FLAT, LIM_MINMOD, LIM_MC, LIM_WENOZ = 0, 1, 2, 3
BC_PERIODIC, BC_OUTFLOW = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle library with g++ (no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-shared",
                           "-fPIC", _SRC, "-o", tmp])
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("dx", ctypes.c_double * 3),
                ("gamma", ctypes.c_double), ("glm_alpha", ctypes.c_double),
                ("rho_floor", ctypes.c_double), ("p_floor", ctypes.c_double),
                ("limiter", ctypes.c_int), ("bc", ctypes.c_int * 6), ("rk_order", ctypes.c_int)]


@dataclass
class Grid:
    """Problem description shared by every oracle call."""
    n: tuple  # (nx, ny, nz)
    dx: tuple = (1.0, 1.0, 1.0)
    gamma: float = 5.0 / 3.0
    glm_alpha: float = 0.1
    rho_floor: float = 1e-12
    p_floor: float = 1e-12
    limiter: int = LIM_MC
    bc: tuple = (BC_PERIODIC,) * 6
    cfl: float = 0.8
    rk_order: int = 2

    @property
    def ghost(self) -> int:
        return 3 if self.limiter == LIM_WENOZ else 2

    def c(self) -> _Params:
        p = _Params()
        for d in range(3):
            p.n[d] = int(self.n[d])
            p.dx[d] = float(self.dx[d])
        p.gamma, p.glm_alpha = self.gamma, self.glm_alpha
        p.rho_floor, p.p_floor = self.rho_floor, self.p_floor
        p.limiter = int(self.limiter)
        for s in range(6):
            p.bc[s] = int(self.bc[s])
        p.rk_order = int(self.rk_order)
        return p

    @property
    def shape(self):
        nx, ny, nz = self.n
        return (9, nz, ny, nx)

    @property
    def ncell(self) -> int:
        return int(np.prod(self.n))


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        P = ctypes.POINTER(_Params)
        LL = ctypes.POINTER(ctypes.c_longlong)
        L = ctypes.c_long
        _lib.orc_prim_to_cons.argtypes = [D, D, L, ctypes.c_double]
        _lib.orc_cons_to_prim.argtypes = [P, D, D, L, LL]
        _lib.orc_fast_speed.argtypes = [D, D, L, ctypes.c_int, ctypes.c_double]
        _lib.orc_interface_flux.argtypes = [D, D, D, L, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double]
        _lib.orc_limited_slope.argtypes = [D, D, D, L, ctypes.c_int]
        _lib.orc_wenoz_face.argtypes = [D, D, L]
        _lib.orc_fill_ghosts.argtypes = [P, D, D]
        _lib.orc_max_speed.argtypes = [P, D, LL]
        _lib.orc_max_speed.restype = ctypes.c_double
        _lib.orc_stage.argtypes = [P, D, D, ctypes.c_double, ctypes.c_double, ctypes.c_int, D,
                                   LL]
        _lib.orc_run.argtypes = [P, D, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, D, D, LL]
        _lib.orc_run.restype = ctypes.c_double
        _lib.orc_run_jvp.argtypes = [P, D, D, ctypes.c_int, D, D]
        _lib.orc_conserved_sums.argtypes = [P, D, D]
        _lib.orc_stage_padded.argtypes = [P, D, D, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int, D]
        _lib.orc_ct_run.argtypes = [P, D, D, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, D, D, LL]
        _lib.orc_ct_run.restype = ctypes.c_double
        _lib.orc_ct_divb.argtypes = [P, D, D]
        _lib.orc_ct_stage1.argtypes = [P, D, D, ctypes.c_double, ctypes.c_double, D, D]
        _lib.orc_ct_edge_emf.argtypes = [D, D, L]
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def prim_to_cons(V: np.ndarray, gamma: float) -> np.ndarray:
    V = _f64(V)
    U = np.empty_like(V)
    lib().orc_prim_to_cons(_d(V), _d(U), V[0].size, gamma)
    return U


def cons_to_prim(U: np.ndarray, grid: Grid):
    """Returns (V, (rho_floor_hits, p_floor_hits))."""
    U = _f64(U)
    V = np.empty_like(U)
    cnt = (ctypes.c_longlong * 2)()
    p = grid.c()
    lib().orc_cons_to_prim(ctypes.byref(p), _d(U), _d(V), U[0].size, cnt)
    return V, (cnt[0], cnt[1])


def fast_speed(V: np.ndarray, d: int, gamma: float) -> np.ndarray:
    V = _f64(V)
    out = np.empty(V[0].shape)
    lib().orc_fast_speed(_d(V), _d(out), V[0].size, d, gamma)
    return out


def interface_flux(VL: np.ndarray, VR: np.ndarray, d: int, ch: float,
                   gamma: float) -> np.ndarray:
    """GLM + HLLD flux for face pairs; VL, VR of shape (9, nface)."""
    VL, VR = _f64(VL), _f64(VR)
    F = np.empty_like(VL)
    lib().orc_interface_flux(_d(VL), _d(VR), _d(F), VL[0].size, d, ch, gamma)
    return F


def limited_slope(dm, dp, lim: int) -> np.ndarray:
    dm, dp = _f64(dm), _f64(dp)
    out = np.empty_like(dm)
    lib().orc_limited_slope(_d(dm), _d(dp), _d(out), dm.size, lim)
    return out


def wenoz_face(f: np.ndarray) -> np.ndarray:
    """WENO-Z value at x_{i+1/2} biased towards cell i from f of shape
    (5, n) = values at cells i-2 .. i+2."""
    f = _f64(f)
    out = np.empty(f.shape[1])
    lib().orc_wenoz_face(_d(f), _d(out), f.shape[1])
    return out


def fill_ghosts(U: np.ndarray, grid: Grid) -> np.ndarray:
    U = _f64(U)
    g = [grid.ghost if n > 1 else 0 for n in grid.n]
    nx, ny, nz = grid.n
    out = np.empty((9, nz + 2 * g[2], ny + 2 * g[1], nx + 2 * g[0]))
    p = grid.c()
    lib().orc_fill_ghosts(ctypes.byref(p), _d(U), _d(out))
    return out


def max_speed(U: np.ndarray, grid: Grid) -> float:
    U = _f64(U)
    p = grid.c()
    return lib().orc_max_speed(ctypes.byref(p), _d(U), None)


def cfl_dt(U: np.ndarray, grid: Grid):
    """(dt, c_h) of the CFL rule: c_h = max speed, dt = cfl / (c_h sum 1/dx_d)."""
    ch = max_speed(U, grid)
    inv = sum(1.0 / grid.dx[d] for d in range(3) if grid.n[d] > 1)
    return grid.cfl / (ch * inv), ch


def stage(W: np.ndarray, grid: Grid, dt: float, ch: float, stage_no: int,
          Un: np.ndarray | None = None):
    W = _f64(W)
    out = np.empty_like(W)
    cnt = (ctypes.c_longlong * 2)()
    p = grid.c()
    un = _d(_f64(Un)) if Un is not None else None
    lib().orc_stage(ctypes.byref(p), _d(W), un, dt, ch, stage_no, _d(out), cnt)
    return out, (cnt[0], cnt[1])


def stage_padded(Wp: np.ndarray, grid: Grid, dt: float, ch: float, stage_no: int,
                 Un: np.ndarray | None = None, damp: bool = False) -> np.ndarray:
    """One stage on a padded array whose ghost zones the caller filled."""
    Wp = _f64(Wp)
    nx, ny, nz = grid.n
    out = np.empty((9, nz, ny, nx))
    p = grid.c()
    un = _d(_f64(Un)) if Un is not None else None
    lib().orc_stage_padded(ctypes.byref(p), _d(Wp), un, dt, ch, stage_no, int(damp), _d(out))
    return out


@dataclass
class RunResult:
    U: np.ndarray
    t: float
    dts: np.ndarray
    chs: np.ndarray
    floors: tuple = field(default=(0, 0))
    b: np.ndarray | None = None  # constrained transport: face field (3, nz, ny, nx)


def run(U0: np.ndarray, grid: Grid, nsteps: int, t0: float = 0.0, t_end: float = 0.0,
        dts=None, chs=None) -> RunResult:
    """nsteps RK2 steps.  dts/chs: optional frozen sequences (else CFL rule)."""
    U = _f64(U0).copy()
    if dts is None:
        dts = np.zeros(nsteps)
        chs = np.zeros(nsteps)
    else:
        dts = _f64(dts).copy()
        chs = _f64(chs).copy()
    cnt = (ctypes.c_longlong * 2)()
    p = grid.c()
    t = lib().orc_run(ctypes.byref(p), _d(U), nsteps, grid.cfl, t0, t_end, _d(dts), _d(chs),
                      cnt)
    return RunResult(U, t, dts, chs, (cnt[0], cnt[1]))


def run_jvp(U0: np.ndarray, dU0: np.ndarray, grid: Grid, dts, chs):
    """Exact forward-mode derivative of the recorded-dt rollout."""
    U, dU = _f64(U0).copy(), _f64(dU0).copy()
    dts, chs = _f64(dts), _f64(chs)
    p = grid.c()
    lib().orc_run_jvp(ctypes.byref(p), _d(U), _d(dU), len(dts), _d(dts), _d(chs))
    return U, dU


def conserved_sums(U: np.ndarray, grid: Grid) -> np.ndarray:
    U = _f64(U)
    out = np.empty(8)
    p = grid.c()
    lib().orc_conserved_sums(ctypes.byref(p), _d(U), _d(out))
    return out


# ----------------------------------------------------- constrained transport --
# Face-field arrays have shape (3, nz, ny, nx): component d on each cell's
# lower d-face.  Three active dimensions, periodic boundaries.

def ct_run(U0: np.ndarray, b0: np.ndarray, grid: Grid, nsteps: int, t0: float = 0.0,
           t_end: float = 0.0, dts=None, chs=None) -> RunResult:
    """nsteps constrained-transport steps (RK2, or SSP-RK3 with
    grid.rk_order == 3).  U0's cell-centred B must be the mean of b0's faces."""
    U = _f64(U0).copy()
    b = _f64(b0).copy()
    if dts is None:
        dts = np.zeros(nsteps)
        chs = np.zeros(nsteps)
    else:
        dts = _f64(dts).copy()
        chs = _f64(chs).copy()
    cnt = (ctypes.c_longlong * 2)()
    p = grid.c()
    t = lib().orc_ct_run(ctypes.byref(p), _d(U), _d(b), nsteps, grid.cfl, t0, t_end, _d(dts),
                         _d(chs), cnt)
    return RunResult(U, t, dts, chs, (cnt[0], cnt[1]), b)


def ct_stage1(W: np.ndarray, bw: np.ndarray, grid: Grid, dt: float, ch: float):
    """One first RK stage with constrained transport: (W + dt L, b + dt db/dt)."""
    W, bw = _f64(W), _f64(bw)
    out, bout = np.empty_like(W), np.empty_like(bw)
    p = grid.c()
    lib().orc_ct_stage1(ctypes.byref(p), _d(W), _d(bw), dt, ch, _d(out), _d(bout))
    return out, bout


def ct_divb(b: np.ndarray, grid: Grid) -> np.ndarray:
    """Face divergence per cell, sum_d (b_d(+1/2) - b_d(-1/2)) / dx_d."""
    b = _f64(b)
    out = np.empty(b.shape[1:])
    p = grid.c()
    lib().orc_ct_divb(ctypes.byref(p), _d(b), _d(out))
    return out


def ct_edge_emf(Ea, Fa, Eb, Fb, Ec) -> np.ndarray:
    """CT-contact edge field for arrays of edges: Ea, Fa, Eb, Fb of shape
    (2, n), Ec of shape (2, 2, n) indexed [a side][b side]."""
    Ea, Fa, Eb, Fb, Ec = (np.asarray(x, dtype=np.float64) for x in (Ea, Fa, Eb, Fb, Ec))
    n = Ea.shape[1]
    inp = np.ascontiguousarray(np.concatenate(
        [Ea, Fa, Eb, Fb, Ec.reshape(4, n)], axis=0))
    out = np.empty(n)
    lib().orc_ct_edge_emf(_d(inp), _d(out), n)
    return out
