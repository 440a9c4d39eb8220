"""The maximum wave speed of the FP64 kernels is the exact FP64 maximum,
although they screen cells with an FP32 estimate before the FP64 evaluation.
Checked against the oracle's maximum speed of the same state (to 1e-13,
round-off of two FP64 evaluations) for both places it is computed: the
wave-speed kernel (mhd_dt after mhd_set_state) and the last stage's epilogue
(mhd_dt after mhd_step).  The states make a screening mistake visible: cell
speeds within 1e-7 of each other (a missed maximum would be off by about
that much), low internal energy, the field along an axis with the sound
speed equal to the Alfven speed (cancellations: unreliable estimates,
evaluated exactly), density varying over a decade with the largest momenta
in dense slow cells (a speed estimate built from momenta instead of
velocities would be caught), variables outside the FP32 image range, a
ragged 3-D grid, a 2-D grid and WENO-Z."""
import numpy as np
import pytest

import oracle as orc

pytestmark = pytest.mark.gpu


def _mhd():
    import paper_2510_24175_gb300 as m
    return m


def _prims(kind, n, seed):
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    V = np.zeros((9, nz, ny, nx))

    def near(b, rel=1e-7):
        return b * (1.0 + rel * rng.standard_normal((nz, ny, nx)))

    if kind == "near_uniform":
        for k, b in enumerate([1.0, 0.3, -0.2, 0.1, 0.5, 0.4, -0.3, 1.0]):
            V[k] = near(b)
    elif kind == "low_internal_energy":  # p / (gamma - 1) << kinetic + magnetic
        for k, b in enumerate([1.0, 2.0, -1.5, 0.5, 1.2, -0.8, 0.6, 1e-3]):
            V[k] = near(b)
    elif kind == "aligned_field":  # B along x, gamma p = Bx^2: c_s = c_a in x
        V[0] = near(1.0)
        V[1], V[2], V[3] = near(0.1), near(0.05), near(-0.02)
        V[4] = near(1.0, 1e-9)
        V[7] = near(0.6, 1e-9)  # gamma * p = 1 = Bx^2 (gamma = 5/3)
    elif kind == "heavy_slow":  # the largest momenta sit in dense, slow cells
        V[0] = np.where(rng.random((nz, ny, nx)) < 0.5, 8.0, 0.5)
        V[1] = near(0.0, 0.0) + 0.3 / V[0] + 1e-7 * rng.standard_normal((nz, ny, nx))
        V[2], V[3] = near(0.1), near(-0.05)
        V[4], V[5], V[6] = near(0.3), near(0.2), near(0.1)
        V[7] = near(1.0)
    elif kind == "tiny_values":  # some variables far below the FP32 image range
        for k, b in enumerate([1.0, 0.3, -0.2, 0.1, 0.5, 0.4, -0.3, 1.0]):
            V[k] = near(b)
        mask = rng.random((nz, ny, nx)) < 0.3
        V[3][mask] = 1e-35
        V[6][~mask] = -1e-33
    elif kind == "random":  # density over a decade: momenta and velocities differ
        V[0] = 0.2 * 10.0 ** rng.random((nz, ny, nx))
        V[1:4] = rng.standard_normal((3, nz, ny, nx))
        V[4:7] = 0.7 * rng.standard_normal((3, nz, ny, nx))
        V[7] = 0.1 + rng.random((nz, ny, nx))
    V[8] = 1e-3 * rng.standard_normal((nz, ny, nx))
    return V


def _check(cfg, V, steps, rough=False):
    import torch
    m = _mhd()
    s = m.MHD(cfg)
    s.set_state(torch.from_numpy(V).cuda(), kind=m.MHD_PRIM)
    g = orc.Grid(n=cfg.n, dx=tuple((cfg.xmax[d] - cfg.xmin[d]) / cfg.n[d] for d in range(3)),
                 gamma=cfg.gamma, limiter=cfg.limiter, bc=cfg.bc)
    for k in range(steps + 1):
        if k:
            s.step()
        U = s.get_state().cpu().numpy()
        _, ch = s.dt()
        ref = orc.max_speed(U, g)
        assert abs(ch - ref) <= 1e-13 * ref, (k, ch, ref, (ch - ref) / ref)
        c = s.counters()
        assert c["status"] == 0
        if not rough:
            assert c["rho_floor"] == 0 and c["p_floor"] == 0


@pytest.mark.parametrize("kind", ["near_uniform", "low_internal_energy", "aligned_field",
                                  "heavy_slow", "tiny_values", "random"])
def test_screened_speed_max_is_exact_3d(kind):
    m = _mhd()
    n = (40, 24, 20)
    cfg = m.Config(n=n)
    _check(cfg, _prims(kind, n, seed=11), steps=2, rough=kind == "random")


@pytest.mark.parametrize("kind", ["near_uniform", "random"])
def test_screened_speed_max_is_exact_2d_and_wenoz(kind):
    m = _mhd()
    n = (48, 40, 1)
    _check(m.Config(n=n), _prims(kind, n, seed=12), steps=2, rough=kind == "random")
    n3 = (32, 16, 12)
    _check(m.Config(n=n3, limiter=m.MHD_LIM_WENOZ, rk_order=3), _prims(kind, n3, seed=13),
           steps=1, rough=kind == "random")
