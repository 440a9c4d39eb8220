"""Seeded synthetic inputs: primitive-variable initial conditions and workloads.

This module holds no step of the numerical method.  It returns PRIMITIVE
fields (rho, vx, vy, vz, Bx, By, Bz, p, psi) as float64 arrays of shape
(9, nz, ny, nx), sampled at cell centres x_i = xmin + (i + 1/2) dx, with
psi = 0.  The conservative conversion is done by whichever implementation
consumes them (the CUDA library through ``mhd_set_state(..., MHD_PRIM)``, the
oracle through its own routine).

The problems are the paper's two gPLUTO test problems (Section 4.2: 3-D
Orszag-Tang vortex and a circularly polarised Alfven wave, "an exact nonlinear
solution"), the Brio & Wu (1988) shock tube, a seeded turbulent box, linear
waves with closed-form solutions, and the seeded adjoint perturbation.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

RHO, VX, VY, VZ, BX, BY, BZ, PRS, PSI = range(9)
LIM_FLAT, LIM_MINMOD, LIM_MC, LIM_WENOZ = 0, 1, 2, 3
BC_PERIODIC, BC_OUTFLOW = 0, 1
FP64, FP32 = 0, 1


@dataclass
class Problem:
    """A workload: grid, physics constants, limiter, BCs, step rule."""
    name: str
    n: tuple                      # (nx, ny, nz); n_d == 1 => inactive dimension
    xmin: tuple = (0.0, 0.0, 0.0)
    xmax: tuple = (1.0, 1.0, 1.0)
    gamma: float = 5.0 / 3.0
    cfl: float = 0.8
    limiter: int = LIM_MC
    bc: tuple = (BC_PERIODIC,) * 6
    glm_alpha: float = 0.1
    rho_floor: float = 1e-12
    p_floor: float = 1e-12
    steps: int = 20
    t_end: float = 0.0            # > 0: clamp the last step to reach t_end
    precision: int = FP64
    rk_order: int = 2             # 2: RK2; 3: SSP-RK3
    seed: int = 0
    params: dict = field(default_factory=dict)

    @property
    def dx(self):
        return tuple((self.xmax[d] - self.xmin[d]) / self.n[d] for d in range(3))

    @property
    def ncell(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])

    def centres(self):
        """Cell-centre coordinate arrays (x, y, z), broadcastable to (nz, ny, nx)."""
        nx, ny, nz = self.n
        dx, dy, dz = self.dx
        x = self.xmin[0] + (np.arange(nx) + 0.5) * dx
        y = self.xmin[1] + (np.arange(ny) + 0.5) * dy
        z = self.xmin[2] + (np.arange(nz) + 0.5) * dz
        return x[None, None, :], y[None, :, None], z[:, None, None]

    def prim(self) -> np.ndarray:
        return _GENERATORS[self.params.get("ic", self.name)](self)

    def with_n(self, n) -> "Problem":
        return replace(self, n=tuple(n))


def _empty(pb: Problem) -> np.ndarray:
    nx, ny, nz = pb.n
    return np.zeros((9, nz, ny, nx))


# ----------------------------------------------------------------- problems --
def _brio_wu(pb: Problem) -> np.ndarray:
    """Brio & Wu (1988) shock tube: jump at x = 0.5, Bx = 0.75."""
    V = _empty(pb)
    x, _, _ = pb.centres()
    left = np.broadcast_to(x < 0.5, V[0].shape)
    V[RHO] = np.where(left, 1.0, 0.125)
    V[PRS] = np.where(left, 1.0, 0.1)
    V[BY] = np.where(left, 1.0, -1.0)
    V[BX] = 0.75
    return V


def _orszag_tang(pb: Problem) -> np.ndarray:
    """Orszag-Tang vortex (3-D form: v_z = vz_amp sin 2 pi z; 2-D: v_z = 0)."""
    V = _empty(pb)
    x, y, z = pb.centres()
    b0 = pb.params.get("B0", 1.0 / math.sqrt(4.0 * math.pi))
    vz_amp = pb.params.get("vz_amp", 0.1 if pb.n[2] > 1 else 0.0)
    tp = 2.0 * math.pi
    shape = V[0].shape
    V[RHO] = 25.0 / (36.0 * math.pi)
    V[PRS] = 5.0 / (12.0 * math.pi)
    V[VX] = np.broadcast_to(-np.sin(tp * y), shape)
    V[VY] = np.broadcast_to(np.sin(tp * x), shape)
    V[VZ] = np.broadcast_to(vz_amp * np.sin(tp * z), shape)
    V[BX] = np.broadcast_to(-b0 * np.sin(tp * y), shape)
    V[BY] = np.broadcast_to(b0 * np.sin(2.0 * tp * x), shape)
    return V


def _half_spectrum(n, rng, kmin, kmax, slope, ncomp):
    """Seeded complex Gaussian modes on the half (real-FFT) spectrum grid,
    shape (ncomp, nz, ny, nx//2+1), with shell spectrum E(k) ~ k^slope for
    integer |k| in [kmin, kmax].  Returns (modes, (kz, ky, kx))."""
    nx, ny, nz = n
    kx = np.fft.rfftfreq(nx, 1.0 / nx)
    ky = np.fft.fftfreq(ny, 1.0 / ny) if ny > 1 else np.zeros(1)
    kz = np.fft.fftfreq(nz, 1.0 / nz) if nz > 1 else np.zeros(1)
    K = np.sqrt(kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2)
    dim = sum(1 for m in n if m > 1)
    # shell spectrum E(k) ~ k^slope  =>  per-mode amplitude ~ k^{(slope - (dim-1))/2}
    amp = np.zeros_like(K)
    mask = (K >= kmin) & (K <= kmax)
    amp[mask] = K[mask] ** ((slope - (dim - 1)) / 2.0)
    modes = np.empty((ncomp,) + K.shape, dtype=np.complex128)
    for c in range(ncomp):
        modes[c].real = rng.standard_normal(K.shape)
        modes[c].imag = rng.standard_normal(K.shape)
        modes[c] *= amp
    return modes, (kz, ky, kx)


def _to_real(modes, n):
    nx, ny, nz = n
    return np.fft.irfftn(modes, s=(nz, ny, nx), axes=(-3, -2, -1))


def _gaussian_field(n, rng, kmin, kmax, slope, ncomp):
    """Real periodic fields (ncomp, nz, ny, nx) with a k^slope shell spectrum."""
    modes, ks = _half_spectrum(n, rng, kmin, kmax, slope, ncomp)
    return np.stack([_to_real(modes[c], n) for c in range(ncomp)]), ks


def _turbulent_box(pb: Problem) -> np.ndarray:
    """rho = 1, p = 0.6; v a seeded Gaussian random field with a k^-2 shell
    spectrum (|k| in [1, 16]) scaled to rms |v| = 0.5; B = (0.2, 0, 0) plus the
    curl of a seeded vector potential of the same spectral shape, rms 0.05
    (divergence-free to round-off: the curl is taken in spectral space)."""
    rng = np.random.default_rng(pb.seed)
    V = _empty(pb)
    V[RHO] = 1.0
    V[PRS] = pb.params.get("p0", 0.6)
    v, _ = _gaussian_field(pb.n, rng, 1, 16, -2.0, 3)
    v *= pb.params.get("v_rms", 0.5) / math.sqrt(np.mean(np.sum(v * v, axis=0)))
    V[VX:VZ + 1] = v
    del v
    Ah, (kz, ky, kx) = _half_spectrum(pb.n, rng, 1, 16, -2.0, 3)
    L = [pb.xmax[d] - pb.xmin[d] for d in range(3)]
    ikx = 2j * math.pi * kx[None, None, :] / L[0]
    iky = 2j * math.pi * ky[None, :, None] / L[1]
    ikz = 2j * math.pi * kz[:, None, None] / L[2]
    b = np.empty((3,) + V[0].shape)
    b[0] = _to_real(iky * Ah[2] - ikz * Ah[1], pb.n)
    b[1] = _to_real(ikz * Ah[0] - ikx * Ah[2], pb.n)
    b[2] = _to_real(ikx * Ah[1] - iky * Ah[0], pb.n)
    del Ah
    brms = math.sqrt(np.mean(np.sum(b * b, axis=0)))
    if brms > 0:
        b *= pb.params.get("b_rms", 0.05) / brms
    V[BX] = pb.params.get("B0x", 0.2) + b[0]
    V[BY] = b[1]
    V[BZ] = b[2]
    return V


def _linear_wave(pb: Problem) -> np.ndarray:
    """Small-amplitude wave along x on a uniform background.

    params: background (rho0, p0, B0 = (bx, by, bz)) and a perturbation
    vector ``dV`` (9 entries) multiplied by amp * sin(2 pi x / Lx).
    """
    V = _empty(pb)
    x, _, _ = pb.centres()
    rho0 = pb.params.get("rho0", 1.0)
    p0 = pb.params.get("p0", 1.0)
    B0 = pb.params.get("B0", (1.0, 0.0, 0.0))
    amp = pb.params.get("amp", 1e-6)
    dV = np.asarray(pb.params["dV"], dtype=np.float64)
    L = pb.xmax[0] - pb.xmin[0]
    s = np.broadcast_to(np.sin(2.0 * math.pi * (x - pb.xmin[0]) / L), V[0].shape)
    V[RHO] = rho0
    V[PRS] = p0
    V[BX], V[BY], V[BZ] = B0
    for k in range(9):
        if dV[k] != 0.0:
            V[k] = V[k] + amp * dV[k] * s
    return V


def _uniform(pb: Problem) -> np.ndarray:
    V = _empty(pb)
    for k, val in enumerate(pb.params["V0"]):
        V[k] = val
    return V


def _random_smooth(pb: Problem) -> np.ndarray:
    """Seeded smooth positive state with all 9 variables varying (psi too),
    for conservation and parity tests."""
    rng = np.random.default_rng(pb.seed)
    V = _empty(pb)
    f, _ = _gaussian_field(pb.n, rng, 1, 4, -2.0, 9)
    f /= np.maximum(np.sqrt(np.mean(f * f, axis=(1, 2, 3), keepdims=True)), 1e-300)
    V[RHO] = 1.0 + 0.3 * np.tanh(f[0])
    V[VX:VZ + 1] = 0.4 * f[1:4]
    V[BX:BZ + 1] = 0.5 * f[4:7] + np.array([0.3, -0.2, 0.1])[:, None, None, None]
    V[PRS] = 1.0 + 0.3 * np.tanh(f[7])
    V[PSI] = 0.05 * f[8] * pb.params.get("psi_amp", 1.0)
    return V


_GENERATORS = {
    "brio_wu": _brio_wu,
    "orszag_tang": _orszag_tang,
    "turbulent": _turbulent_box,
    "linear_wave": _linear_wave,
    "uniform": _uniform,
    "random_smooth": _random_smooth,
}


# ---------------------------------------------------------- named workloads --
def brio_wu(nx: int = 1024) -> Problem:
    """1-D Brio-Wu, gamma = 2, minmod, CFL 0.8, outflow, to t = 0.1."""
    return Problem("brio_wu", (nx, 1, 1), gamma=2.0, limiter=LIM_MINMOD,
                   bc=(BC_OUTFLOW,) * 6, cfl=0.8, steps=100000, t_end=0.1)


def orszag_tang_3d(n: int = 256, steps: int = 20) -> Problem:
    """3-D Orszag-Tang, periodic [0,1]^3, gamma = 5/3, MC, FP64."""
    return Problem("orszag_tang", (n, n, n), limiter=LIM_MC, steps=steps)


def turbulent_box(n: int = 512, steps: int = 50, seed: int = 3,
                  precision: int = FP32) -> Problem:
    """Seeded turbulent box, periodic, FP32 bulk."""
    return Problem("turbulent", (n, n, n), limiter=LIM_MC, steps=steps, seed=seed,
                   precision=precision)


def orszag_tang_2d(n: int = 512, steps: int = 200) -> Problem:
    """2-D Orszag-Tang (n x n x 1), used by the adjoint workload."""
    return Problem("orszag_tang", (n, n, 1), limiter=LIM_MC, steps=steps)


def adjoint_perturbation(pb: Problem, seed: int = 4, rms: float = 1e-3,
                         kmax: int = 8) -> np.ndarray:
    """Seeded smooth velocity perturbation (vx, vy) with modes |k| <= kmax,
    scaled to rms |dv| = rms.  Shape (2, nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    f, _ = _gaussian_field(pb.n, rng, 1, kmax, -2.0, 2)
    f *= rms / math.sqrt(np.mean(np.sum(f * f, axis=0)))
    return f


def random_directions(shape, count: int, seed: int = 4) -> np.ndarray:
    """Seeded unit-norm random directions, shape (count,) + shape."""
    rng = np.random.default_rng(seed + 1000)
    d = rng.standard_normal((count,) + tuple(shape))
    d /= np.sqrt(np.sum(d.reshape(count, -1) ** 2, axis=1)).reshape((count,) + (1,) * len(shape))
    return d


def ensemble_sizes(count: int = 64, seed: int = 5):
    """Box edges drawn from {32, 48, 64, 96, 128} and B0 from U[0.1, 0.5]."""
    rng = np.random.default_rng(seed)
    edges = rng.choice([32, 48, 64, 96, 128], size=count)
    b0 = rng.uniform(0.1, 0.5, size=count)
    return [int(e) for e in edges], [float(b) for b in b0]


def random_face_states(count: int, seed: int, degenerate: str | None = None) -> tuple:
    """Seeded random primitive face pairs (VL, VR), each (9, count), positive
    rho and p.  ``degenerate`` selects special families: 'bn0' (B_n = 0),
    'bt0' (B_t = 0), 'b0' (B = 0), 'vacuum' (rho, p ~ 1e-6), 'equal' (VL = VR)."""
    rng = np.random.default_rng(seed)

    def one():
        V = np.empty((9, count))
        V[RHO] = np.exp(rng.uniform(-2.0, 2.0, count))
        V[VX:VZ + 1] = rng.normal(0.0, 1.0, (3, count))
        V[BX:BZ + 1] = rng.normal(0.0, 1.0, (3, count))
        V[PRS] = np.exp(rng.uniform(-2.0, 2.0, count))
        V[PSI] = rng.normal(0.0, 0.1, count)
        return V

    VL, VR = one(), one()
    if degenerate == "equal":
        VR = VL.copy()
    elif degenerate == "bn0":
        VL[BX] = 0.0
        VR[BX] = 0.0
        VL[PSI] = 0.0
        VR[PSI] = 0.0
    elif degenerate == "bt0":
        VL[BY:BZ + 1] = 0.0
        VR[BY:BZ + 1] = 0.0
    elif degenerate == "b0":
        VL[BX:BZ + 1] = 0.0
        VR[BX:BZ + 1] = 0.0
        VL[PSI] = 0.0
        VR[PSI] = 0.0
    elif degenerate == "vacuum":
        VL[RHO] *= 1e-6
        VR[RHO] *= 1e-6
        VL[PRS] *= 1e-6
        VR[PRS] *= 1e-6
    return VL, VR
