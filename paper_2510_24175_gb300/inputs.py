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
DIVB_GLM, DIVB_CT = 0, 1


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
    divb: int = DIVB_GLM          # div-B control: GLM cleaning or constrained transport
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

    def faces(self) -> np.ndarray:
        """Staggered magnetic field for constrained transport, shape
        (3, nz, ny, nx): component d on each cell's lower d-face (at
        x_d = xmin_d + i_d dx_d, the other coordinates at cell centres).  The
        cell-centred B of ``prim()`` is the mean of each cell's two faces."""
        return _FACE_GENERATORS[self.params.get("ic", self.name)](self)

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


def _floor_defects(pb: Problem) -> np.ndarray:
    """The smooth random state with seeded defect cells that drive the floor
    branches of cons->prim: ``n_rho`` near-vacuum cells (rho = rho_defect,
    v = 0), ``n_p`` cells with a negative pressure (p = p_defect < 0: their
    total energy is below the kinetic plus magnetic energy), and ``n_cold``
    cold, strongly magnetised, fast cells (p = p_cold, |B| ~ b_cold,
    |v| ~ 1), whose internal energy is a tiny fraction of the total.  Defect
    cells are distinct and at least two cells apart along every axis.
    ``p_base`` scales the background pressure (a cold flow when small)."""
    V = _random_smooth(pb)
    q = pb.params
    V[PRS] *= q.get("p_base", 1.0)
    rng = np.random.default_rng(pb.seed + 1000)
    nx, ny, nz = pb.n
    counts = (q.get("n_rho", 0), q.get("n_p", 0), q.get("n_cold", 0))
    picked = []
    while len(picked) < sum(counts):
        c = (int(rng.integers(nz)), int(rng.integers(ny)), int(rng.integers(nx)))
        if all(max(abs(c[0] - o[0]), abs(c[1] - o[1]), abs(c[2] - o[2])) > 2 for o in picked):
            picked.append(c)
    kinds = [0] * counts[0] + [1] * counts[1] + [2] * counts[2]
    for (k, j, i), kind in zip(picked, kinds):
        if kind == 0:
            V[RHO, k, j, i] = q.get("rho_defect", 1e-5)
            V[VX:VZ + 1, k, j, i] = 0.0
        elif kind == 1:
            V[PRS, k, j, i] = q.get("p_defect", -0.5)
        else:
            V[PRS, k, j, i] = q.get("p_cold", 1e-5)
            b = rng.normal(size=3)
            V[BX:BZ + 1, k, j, i] = q.get("b_cold", 2.0) * b / np.linalg.norm(b)
            v = rng.normal(size=3)
            V[VX:VZ + 1, k, j, i] = v / np.linalg.norm(v)
    return V


def _cold_flow(pb: Problem) -> np.ndarray:
    """A cold, strongly magnetised, highly supersonic uniform flow with small
    seeded smooth perturbations: rho = 1, v = (1, 0.5, 0.2), B = (0.5, 0.3,
    0.1), each with a relative perturbation of rms ``amp`` (default 1e-5), and
    p = p0 (default 1e-4) times (1 + 0.1 tanh f): the internal energy is
    about 2e-4 of the total in every cell."""
    rng = np.random.default_rng(pb.seed)
    q = pb.params
    amp = q.get("amp", 1e-5)
    f, _ = _gaussian_field(pb.n, rng, 1, 4, -2.0, 8)
    f /= np.maximum(np.sqrt(np.mean(f * f, axis=(1, 2, 3), keepdims=True)), 1e-300)
    V = _empty(pb)
    base = (1.0, 1.0, 0.5, 0.2, 0.5, 0.3, 0.1)
    for k in range(7):
        V[k] = base[k] * (1.0 + amp * f[k])
    V[PRS] = q.get("p0", 1e-4) * (1.0 + 0.1 * np.tanh(f[7]))
    return V


# ------------------------------------------- staggered (face) magnetic fields --
def _cell_mean(b: np.ndarray) -> np.ndarray:
    """Cell-centred field = mean of each cell's two faces (periodic)."""
    return np.stack([0.5 * (b[0] + np.roll(b[0], -1, axis=2)),
                     0.5 * (b[1] + np.roll(b[1], -1, axis=1)),
                     0.5 * (b[2] + np.roll(b[2], -1, axis=0))])


def _faces_from_cells(pb: Problem) -> np.ndarray:
    """For fields whose component d does not vary along d (Orszag-Tang,
    plane-parallel states with a constant normal component, z-polarised
    waves in the x-y plane): the face value equals the cell value."""
    V = pb.prim()
    return np.ascontiguousarray(V[BX:BZ + 1])


def _potential_modes(pb: Problem):
    """Seeded Fourier modes of a smooth periodic vector potential on [0,1]^3:
    per component, six (k, amplitude, phase) triples with |k_i| <= 3."""
    rng = np.random.default_rng(pb.seed + 7919)
    modes = []
    for _ in range(3):
        comp = []
        while len(comp) < 6:
            k = rng.integers(-3, 4, size=3)
            if not k.any():
                continue
            amp = pb.params.get("a_amp", 0.08) * rng.standard_normal() / np.linalg.norm(k)
            comp.append((k.astype(np.float64), amp, rng.uniform(0.0, 2.0 * math.pi)))
        modes.append(comp)
    return modes


def _line_integral(comp_modes, c: int, mid, h: float):
    """Exact integral of sum_m a_m sin(2 pi k_m . x + phi_m) along axis c over a
    segment of length h centred at the points ``mid`` (tuple of broadcastable
    x, y, z arrays): h sin(2 pi k . mid + phi) sinc(pi k_c h) per mode."""
    out = 0.0
    for k, a, ph in comp_modes:
        arg = 2.0 * math.pi * (k[0] * mid[0] + k[1] * mid[1] + k[2] * mid[2]) + ph
        u = math.pi * k[c] * h
        sinc = math.sin(u) / u if u != 0.0 else 1.0
        out = out + a * h * sinc * np.sin(arg)
    return out


def _potential_faces(pb: Problem, A=None, mean=None) -> np.ndarray:
    """Face averages of B = B_mean + curl A, each from Stokes' theorem as the
    exact circulation of A around the face divided by its area, so the
    discrete divergence vanishes to round-off.  A: per component a list of
    (integer k, amplitude, phase) modes of sin(2 pi k.x + phase) (default: the
    seeded smooth potential)."""
    nx, ny, nz = pb.n
    dx, dy, dz = pb.dx
    xf = (np.arange(nx) * dx)[None, None, :]
    yf = (np.arange(ny) * dy)[None, :, None]
    zf = (np.arange(nz) * dz)[:, None, None]
    xc, yc, zc = xf + 0.5 * dx, yf + 0.5 * dy, zf + 0.5 * dz
    if A is None:
        A = _potential_modes(pb)
    shape = (nz, ny, nx)
    b = np.zeros((3,) + shape)
    # x-face at x = xf: circulation in the (y, z) plane
    b[0] = ((_line_integral(A[2], 2, (xf, yf + dy, zc), dz)
             - _line_integral(A[2], 2, (xf, yf, zc), dz))
            - (_line_integral(A[1], 1, (xf, yc, zf + dz), dy)
               - _line_integral(A[1], 1, (xf, yc, zf), dy))) / (dy * dz)
    # y-face at y = yf: circulation in the (z, x) plane
    b[1] = ((_line_integral(A[0], 0, (xc, yf, zf + dz), dx)
             - _line_integral(A[0], 0, (xc, yf, zf), dx))
            - (_line_integral(A[2], 2, (xf + dx, yf, zc), dz)
               - _line_integral(A[2], 2, (xf, yf, zc), dz))) / (dz * dx)
    # z-face at z = zf: circulation in the (x, y) plane
    b[2] = ((_line_integral(A[1], 1, (xf + dx, yc, zf), dy)
             - _line_integral(A[1], 1, (xf, yc, zf), dy))
            - (_line_integral(A[0], 0, (xc, yf + dy, zf), dx)
               - _line_integral(A[0], 0, (xc, yf, zf), dx))) / (dx * dy)
    if mean is None:
        mean = pb.params.get("B_mean", (0.3, -0.2, 0.1))
    b += np.asarray(mean, dtype=np.float64)[:, None, None, None]
    return b


def _ct_random(pb: Problem) -> np.ndarray:
    """Seeded smooth state (rho, v, p as the random smooth state, psi = 0)
    with a divergence-free staggered field; cell B = face means."""
    V = _random_smooth(pb)
    V[PSI] = 0.0
    V[BX:BZ + 1] = _cell_mean(_potential_faces(pb))
    return V


def _shock_pair(pb: Problem) -> np.ndarray:
    """Two Brio-Wu shock tubes back to back along ``axis`` (periodic): the
    Brio-Wu left state for s < 0.25 or s >= 0.75, the right state between;
    normal field 0.75; the transverse field in the next axis (cyclic)."""
    a = pb.params.get("axis", 0)
    V = _empty(pb)
    s = pb.centres()[a]
    inner = np.broadcast_to((s >= 0.25) & (s < 0.75), V[0].shape)
    V[RHO] = np.where(inner, 0.125, 1.0)
    V[PRS] = np.where(inner, 0.1, 1.0)
    V[BX + (a + 1) % 3] = np.where(inner, -1.0, 1.0)
    V[BX + a] = 0.75
    return V


def _field_loop(pb: Problem) -> np.ndarray:
    """Weak magnetic field loop (Gardiner & Stone 2005) advected by a uniform
    flow: A_z = A0 max(R - r, 0) about the box centre, rho = p = 1."""
    V = _empty(pb)
    V[RHO] = 1.0
    V[PRS] = 1.0
    vel = pb.params.get("v", (1.0, 0.5, 0.0))
    for d in range(3):
        V[VX + d] = vel[d]
    V[BX:BZ + 1] = _cell_mean(_field_loop_faces(pb))
    return V


def _field_loop_faces(pb: Problem) -> np.ndarray:
    nx, ny, nz = pb.n
    dx, dy, _ = pb.dx
    a0 = pb.params.get("A0", 1e-3)
    R = pb.params.get("R", 0.3)

    def az(x, y):
        r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2)
        return a0 * np.maximum(R - r, 0.0)

    xf = (np.arange(nx) * dx)[None, None, :]
    yf = (np.arange(ny) * dy)[None, :, None]
    b = np.zeros((3, nz, ny, nx))
    b[0] = np.broadcast_to((az(xf, yf + dy) - az(xf, yf)) / dy, b[0].shape)
    b[1] = np.broadcast_to(-(az(xf + dx, yf) - az(xf, yf)) / dx, b[1].shape)
    return b


def _cpa_geometry(pb: Problem):
    """Wave vector (integer multiples of 2 pi on [0,1]^3), unit vectors of the
    circularly polarised Alfven wave, and its parameters."""
    kint = np.asarray(pb.params.get("k", (1, 1, 1)), dtype=np.float64)
    khat = kint / np.linalg.norm(kint)
    # e1: a unit vector normal to k (in the plane of k and the axis least
    # aligned with it); e2 = k x e1
    axis = np.zeros(3)
    axis[int(np.argmin(np.abs(khat)))] = 1.0
    e1 = axis - khat * (axis @ khat)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(khat, e1)
    amp = pb.params.get("amp", 0.1)
    bpar = pb.params.get("B0", 1.0)
    rho0 = pb.params.get("rho0", 1.0)
    return kint, khat, e1, e2, amp, bpar, rho0


def _cpa(pb: Problem) -> np.ndarray:
    """Circularly polarised Alfven wave (the paper's second gPLUTO test, an
    exact nonlinear solution; set-up of Toth 2000): uniform rho and p,
    B = B0 k + A (sin phi e1 + cos phi e2), v = -(B - B0 k)/sqrt(rho), phase
    phi = 2 pi k.x - omega t travelling along k at v_A = B0/sqrt(rho).  The
    magnetic pressure is uniform, so the wave keeps its shape.  With GLM the
    cell B is sampled at centres; the CT face field (``faces()``) holds exact
    face averages from the vector potential and the cell B is their mean."""
    kint, khat, e1, e2, amp, bpar, rho0 = _cpa_geometry(pb)
    V = _empty(pb)
    x, y, z = pb.centres()
    t = pb.params.get("t", 0.0)
    vA = bpar / math.sqrt(rho0)
    ph = 2.0 * math.pi * (kint[0] * x + kint[1] * y + kint[2] * z
                          - np.linalg.norm(kint) * vA * t)
    sn = np.broadcast_to(np.sin(ph), V[0].shape)
    cs = np.broadcast_to(np.cos(ph), V[0].shape)
    V[RHO] = rho0
    V[PRS] = pb.params.get("p0", 0.1)
    for c in range(3):
        dB = amp * (sn * e1[c] + cs * e2[c])
        V[BX + c] = bpar * khat[c] + dB
        V[VX + c] = -dB / math.sqrt(rho0)
    if pb.divb == DIVB_CT:
        V[BX:BZ + 1] = _cell_mean(_cpa_faces(pb))
    return V


def _cpa_faces(pb: Problem) -> np.ndarray:
    """Exact face averages of the CPA field: dB = curl a with
    a = (A / |2 pi k|) (sin phi e1 + cos phi e2), plus the uniform B0 k."""
    kint, khat, e1, e2, amp, bpar, _ = _cpa_geometry(pb)
    t = pb.params.get("t", 0.0)
    vA = bpar / math.sqrt(pb.params.get("rho0", 1.0))
    kn = np.linalg.norm(kint)
    ph0 = -2.0 * math.pi * kn * vA * t
    scale = amp / (2.0 * math.pi * kn)
    A = [[(kint, scale * e1[c], ph0), (kint, scale * e2[c], ph0 + 0.5 * math.pi)]
         for c in range(3)]
    return _potential_faces(pb, A=A, mean=bpar * khat)


def _alfven_oblique(pb: Problem) -> np.ndarray:
    """Linear Alfven wave travelling along (1, 1, 0)/sqrt 2 with wave vector
    2 pi (1, 1, 0): background B0 = |B0| (1, 1, 0)/sqrt 2, z-polarised
    perturbation dv_z = A sin(2 pi (x + y)), dB_z = -A sqrt(rho) sin(...)."""
    V = _empty(pb)
    x, y, _ = pb.centres()
    rho0 = pb.params.get("rho0", 1.0)
    amp = pb.params.get("amp", 1e-6)
    bpar = pb.params.get("B0", 1.0)
    t = pb.params.get("t", 0.0)
    vA = bpar / math.sqrt(rho0)
    ph = 2.0 * math.pi * (x + y - math.sqrt(2.0) * vA * t)
    sn = np.broadcast_to(np.sin(ph), V[0].shape)
    V[RHO] = rho0
    V[PRS] = pb.params.get("p0", 1.0)
    V[BX] = bpar / math.sqrt(2.0)
    V[BY] = bpar / math.sqrt(2.0)
    V[VZ] = amp * sn
    V[BZ] = -amp * math.sqrt(rho0) * sn
    return V


_GENERATORS = {
    "brio_wu": _brio_wu,
    "orszag_tang": _orszag_tang,
    "turbulent": _turbulent_box,
    "linear_wave": _linear_wave,
    "uniform": _uniform,
    "random_smooth": _random_smooth,
    "floor_defects": _floor_defects,
    "cold_flow": _cold_flow,
    "ct_random": _ct_random,
    "shock_pair": _shock_pair,
    "field_loop": _field_loop,
    "alfven_oblique": _alfven_oblique,
    "cpa": _cpa,
}

_FACE_GENERATORS = {
    "orszag_tang": _faces_from_cells,
    "uniform": _faces_from_cells,
    "shock_pair": _faces_from_cells,
    "alfven_oblique": _faces_from_cells,
    "ct_random": _potential_faces,
    "field_loop": _field_loop_faces,
    "cpa": _cpa_faces,
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


def orszag_tang_3d_ct(n: int = 256, steps: int = 20, limiter: int = LIM_MC,
                      rk_order: int = 2) -> Problem:
    """3-D Orszag-Tang with constrained transport (periodic [0,1]^3)."""
    return Problem("orszag_tang", (n, n, n), limiter=limiter, steps=steps, rk_order=rk_order,
                   divb=DIVB_CT)


def ct_random(n, seed: int = 11) -> Problem:
    """Seeded smooth state with a divergence-free staggered field."""
    n = tuple(n) if not isinstance(n, int) else (n, n, n)
    return Problem("ct_random", n, limiter=LIM_MC, seed=seed, divb=DIVB_CT)


def shock_pair(n_long: int, n_trans: int = 4, axis: int = 0) -> Problem:
    """Two back-to-back Brio-Wu tubes along ``axis`` on a periodic 3-D grid
    (gamma = 2, minmod), constant across the other two axes."""
    n = [n_trans] * 3
    n[axis] = n_long
    return Problem("shock_pair", tuple(n), gamma=2.0, limiter=LIM_MINMOD, divb=DIVB_CT,
                   params={"axis": axis})


def field_loop(n: int, nz: int = 2, v=(1.0, 0.5, 0.0)) -> Problem:
    """Weak field loop advected diagonally (periodic [0,1]^2 x nz planes)."""
    return Problem("field_loop", (n, n, nz), limiter=LIM_MC, divb=DIVB_CT,
                   params={"v": tuple(v)})


def cpa_wave(n: int, k=(1, 1, 1), divb: int = DIVB_GLM, limiter: int = LIM_MC,
             rk_order: int = 2) -> Problem:
    """Circularly polarised Alfven wave on a periodic n^3 grid, wave vector
    2 pi k, amplitude 0.1, B0 = 1, rho = 1, p = 0.1, gamma = 5/3; one period
    is 1 / |k|."""
    return Problem("cpa", (n, n, n), limiter=limiter, rk_order=rk_order, divb=divb,
                   params={"k": tuple(k)})


def alfven_oblique(n: int, nz: int = 2, amp: float = 1e-6) -> Problem:
    """Oblique linear Alfven wave in the x-y plane (periodic, nz planes)."""
    return Problem("alfven_oblique", (n, n, nz), limiter=LIM_MC, divb=DIVB_CT,
                   params={"amp": amp})


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
