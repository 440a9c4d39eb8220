"""Pins of the oracle's full RK2 step against what the mathematics fixes:
ghost fill vs numpy padding, uniform-state preservation, exact conservation
under periodic boundaries, translation / axis-permutation / reflection /
point-inversion symmetry, closed-form boundary fluxes of the Brio-Wu tube,
the decoupled linear (B_x, psi) subsystem against an independent upwind
scheme, second-order convergence of linear waves to their closed forms, the
dual-number JVP against central finite differences, and one RK2 (PLM) and
one SSP-RK3 (WENO-Z) step, every stage and the damping, rebuilt in numpy
from the separately pinned pieces.
"""
import math

import numpy as np
import pytest

import oracle as orc
from paper_2510_24175_gb300 import inputs
from paper_2510_24175_gb300.inputs import Problem

RHO, VX, VY, VZ, BX, BY, BZ, PRS, PSI = range(9)


def grid_of(pb: Problem) -> orc.Grid:
    return orc.Grid(n=pb.n, dx=pb.dx, gamma=pb.gamma, glm_alpha=pb.glm_alpha,
                    rho_floor=pb.rho_floor, p_floor=pb.p_floor, limiter=pb.limiter,
                    bc=pb.bc, cfl=pb.cfl, rk_order=pb.rk_order)


def cons_of(pb: Problem) -> np.ndarray:
    return orc.prim_to_cons(pb.prim(), pb.gamma)


# ------------------------------------------------------------------ pieces --
def test_prim_cons_hand_value_and_roundtrip():
    V = np.zeros((9, 1))
    V[:, 0] = [2.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 1.0, 0.25]
    U = orc.prim_to_cons(V, 5.0 / 3.0)
    # E = p/(g-1) + rho v^2/2 + B^2/2 = 1.5 + 1 + 0.5
    np.testing.assert_array_equal(U[:, 0], [2.0, 2.0, 0, 0, 0, 1.0, 0, 3.0, 0.25])
    pb = Problem("random_smooth", (6, 5, 4), seed=3)
    Vr = pb.prim()
    V2, floors = orc.cons_to_prim(orc.prim_to_cons(Vr, pb.gamma), grid_of(pb))
    np.testing.assert_allclose(V2, Vr, rtol=1e-13, atol=1e-14)
    assert floors == (0, 0)


def test_pressure_floor_counted():
    V = np.zeros((9, 2))
    V[RHO] = 1.0
    V[PRS] = [1.0, 1.0]
    U = orc.prim_to_cons(V, 5.0 / 3.0)
    U[PRS, 1] = -1.0  # negative internal energy
    g = orc.Grid(n=(2, 1, 1))
    V2, floors = orc.cons_to_prim(U, g)
    assert floors == (0, 1)
    assert V2[PRS, 1] == g.p_floor


@pytest.mark.parametrize("bc,mode", [(orc.BC_PERIODIC, "wrap"), (orc.BC_OUTFLOW, "edge")])
def test_ghost_fill_matches_numpy_pad(bc, mode):
    rng = np.random.default_rng(0)
    for n in [(7, 5, 4), (6, 1, 1), (5, 4, 1)]:
        U = rng.standard_normal((9, n[2], n[1], n[0]))
        g = orc.Grid(n=n, bc=(bc,) * 6)
        pad = [(0, 0)] + [(2, 2) if n[d] > 1 else (0, 0) for d in (2, 1, 0)]
        np.testing.assert_array_equal(orc.fill_ghosts(U, g), np.pad(U, pad, mode=mode))


def test_uniform_state_preserved_exactly():
    for bc in (orc.BC_PERIODIC, orc.BC_OUTFLOW):
        pb = Problem("uniform", (6, 5, 4), bc=(bc,) * 6,
                     params={"V0": [1.3, 0.2, -0.4, 0.1, 0.5, -0.3, 0.7, 0.9, 0.0]})
        U0 = cons_of(pb)
        r = orc.run(U0, grid_of(pb), 3)
        np.testing.assert_allclose(r.U, U0, rtol=2e-15, atol=2e-15)


def test_uniform_state_dt_closed_form():
    V0 = [1.3, 0.2, -0.4, 0.1, 0.5, -0.3, 0.7, 0.9, 0.0]
    pb = Problem("uniform", (6, 5, 4), params={"V0": V0})
    g = grid_of(pb)
    dt, ch = orc.cfl_dt(cons_of(pb), g)
    rho, p, B = V0[0], V0[7], np.array(V0[4:7])
    gam = pb.gamma
    best = 0.0
    for d in range(3):
        a2, ca2 = gam * p / rho, B @ B / rho
        can2 = B[d] ** 2 / rho
        cf = math.sqrt(0.5 * (a2 + ca2 + math.sqrt((a2 + ca2) ** 2 - 4 * a2 * can2)))
        best = max(best, abs(V0[1 + d]) + cf)
    assert ch == pytest.approx(best, rel=1e-14)
    assert dt == pytest.approx(pb.cfl / (best * (6 + 5 + 4)), rel=1e-14)


# ---------------------------------------------------------- conservation --
def test_periodic_conservation_roundoff():
    pb = Problem("random_smooth", (12, 10, 8), seed=5)
    g = grid_of(pb)
    U0 = cons_of(pb)
    s0 = orc.conserved_sums(U0, g)
    r = orc.run(U0, g, 6)
    s1 = orc.conserved_sums(r.U, g)
    scale = np.maximum(np.abs(s0), orc.conserved_sums(np.abs(U0), g))
    assert np.all(np.abs(s1 - s0) <= 1e-13 * scale), (s1 - s0) / scale
    assert r.floors == (0, 0)


# ---------------------------------------------------------------- symmetry --
def test_translation_invariance_bitwise():
    pb = Problem("random_smooth", (8, 6, 5), seed=7)
    g = grid_of(pb)
    U0 = cons_of(pb)
    sh = (1, 2, 3)  # (z, y, x) shifts
    a = orc.run(U0, g, 3).U
    b = orc.run(np.roll(U0, sh, axis=(1, 2, 3)), g, 3).U
    np.testing.assert_array_equal(np.roll(a, sh, axis=(1, 2, 3)), b)


def _cycle_axes(U):
    """Relabel axes: old x -> new y, old y -> new z, old z -> new x, moving
    vector components the same way.  Arrays are (v, z, y, x), so the new
    (z, y, x) axes are the old (y, x, z) axes."""
    T = np.transpose(U, (0, 2, 3, 1))
    W = np.empty((9,) + T.shape[1:])
    for k in (RHO, PRS, PSI):
        W[k] = T[k]
    for base in (VX, BX):
        W[base + 1] = T[base + 0]
        W[base + 2] = T[base + 1]
        W[base + 0] = T[base + 2]
    return W


def test_axis_permutation():
    pb = Problem("random_smooth", (8, 6, 5), seed=8)
    g = grid_of(pb)
    U0 = cons_of(pb)
    a = orc.run(U0, g, 3).U
    W0 = _cycle_axes(U0)
    nz, ny, nx = W0.shape[1:]
    pb2 = pb.with_n((nx, ny, nz))
    b = orc.run(W0, grid_of(pb2), 3).U
    np.testing.assert_allclose(b, _cycle_axes(a), rtol=1e-12, atol=1e-13)


def test_reflection_x():
    """x -> -x with (m_x, B_x) negated is a symmetry of the scheme."""
    pb = Problem("random_smooth", (8, 6, 5), seed=9)
    g = grid_of(pb)
    U0 = cons_of(pb)
    M = np.array([1, -1, 1, 1, -1, 1, 1, 1, 1.0])[:, None, None, None]
    a = orc.run(U0, g, 3).U
    b = orc.run(M * U0[:, :, :, ::-1], g, 3).U
    np.testing.assert_allclose(b, M * a[:, :, :, ::-1], rtol=1e-12, atol=1e-13)


def test_orszag_tang_point_symmetry():
    """The OT ICs are invariant under r -> -r with v, B -> -v, -B; so is the
    scheme (periodic, cell-centred grid: index i -> N-1-i)."""
    pb = inputs.orszag_tang_3d(16, steps=4)
    g = grid_of(pb)
    r = orc.run(cons_of(pb), g, pb.steps)
    U = r.U
    inv = U[:, ::-1, ::-1, ::-1]
    sym = np.array([1, -1, -1, -1, -1, -1, -1, 1, 1.0])[:, None, None, None]
    scale = np.max(np.abs(U), axis=(1, 2, 3), keepdims=True) + 1e-300
    assert np.max(np.abs(U - sym * inv) / scale) < 1e-12
    assert r.floors == (0, 0)


# ------------------------------------------------------------ Brio-Wu tube --
def test_brio_wu_boundary_fluxes_closed_form():
    """Until the outermost waves reach the ends, the outflow boundary fluxes
    are the physical fluxes of the two initial states: mass, energy and B_y
    are conserved, the x-momentum grows at pt_L - pt_R and the y-momentum at
    -Bx (By_L - By_R) (the fluxes rho u^2 + pt - Bx^2 and rho u v - Bx By)."""
    pb = inputs.brio_wu(256)
    g = grid_of(pb)
    U0 = cons_of(pb)
    r = orc.run(U0, g, 100000, t_end=pb.t_end)
    assert r.t == pytest.approx(0.1, abs=1e-15)
    s0, s1 = orc.conserved_sums(U0, g), orc.conserved_sums(r.U, g)
    # order: rho, mx, my, mz, E, Bx, By, Bz
    for q in (0, 3, 4, 5, 6, 7):
        assert abs(s1[q] - s0[q]) < 1e-12, q
    assert s1[2] - s0[2] == pytest.approx(-0.75 * 2.0 * 0.1, rel=1e-12)
    pt_l = 1.0 + 0.5 * (0.75 ** 2 + 1.0)
    pt_r = 0.1 + 0.5 * (0.75 ** 2 + 1.0)
    assert s1[1] - s0[1] == pytest.approx((pt_l - pt_r) * 0.1, rel=1e-12)
    V, fl = orc.cons_to_prim(r.U, g)
    assert fl == (0, 0) and r.floors == (0, 0)
    assert V[RHO].min() > 0.1 and V[PRS].min() > 0.05
    # far-field states untouched up to the exponentially small numerical
    # tails of the discrete domain of dependence
    np.testing.assert_allclose(V[RHO, 0, 0, :5], 1.0, rtol=1e-10)
    np.testing.assert_allclose(V[RHO, 0, 0, -5:], 0.125, rtol=1e-10)


# ------------------------------------------------------- GLM subsystem pin --
def test_glm_subsystem_matches_linear_upwind():
    """With a flat (first-order) reconstruction the (B_x, psi) pair obeys the
    linear system B_t + psi_x = 0, psi_t + ch^2 B_x = 0 decoupled from the
    other variables: w+- = psi +- ch B_x are upwind-advected at +-ch by
    two-stage RK2, then psi is damped by exp(-alpha ch dt / dx)."""
    n = 32
    x = (np.arange(n) + 0.5) / n
    pb = Problem("uniform", (n, 1, 1), limiter=orc.LIM_FLAT, glm_alpha=0.3,
                 params={"V0": [1.0, 0.1, 0.0, 0.0, 0.0, 0.2, 0.0, 1.0, 0.0]})
    V = pb.prim()
    V[BX, 0, 0, :] = 0.1 * np.sin(2 * np.pi * x)
    V[PSI, 0, 0, :] = 0.05 * np.cos(4 * np.pi * x)
    g = grid_of(pb)
    U0 = orc.prim_to_cons(V, pb.gamma)
    ch, dt, dx = 2.0, 0.01, 1.0 / n
    nsteps = 3
    r = orc.run(U0, g, nsteps, dts=[dt] * nsteps, chs=[ch] * nsteps)

    b = V[BX, 0, 0].copy()
    psi = V[PSI, 0, 0].copy()
    wp, wm = psi + ch * b, psi - ch * b

    def L(wp, wm):
        # upwind: w+ moves right (flux ch w+ from left cell), w- moves left
        return (-ch * (wp - np.roll(wp, 1)) / dx, ch * (np.roll(wm, -1) - wm) / dx)

    for _ in range(nsteps):
        a1, b1 = L(wp, wm)
        p1, m1 = wp + dt * a1, wm + dt * b1
        a2, b2 = L(p1, m1)
        wp, wm = 0.5 * (wp + p1 + dt * a2), 0.5 * (wm + m1 + dt * b2)
        b = (wp - wm) / (2 * ch)
        psi = (wp + wm) / 2 * math.exp(-0.3 * ch * dt / dx)
        wp, wm = psi + ch * b, psi - ch * b
    np.testing.assert_allclose(r.U[BX, 0, 0], b, rtol=0, atol=1e-14)
    np.testing.assert_allclose(r.U[PSI, 0, 0], psi, rtol=0, atol=1e-14)


# -------------------------------------------------------------- convergence --
def _wave_problem(kind, n, limiter):
    rho0, p0, gam = 1.0, 1.0, 5.0 / 3.0
    if kind == "alfven":  # B0 = (1,0,0): v_A = 1, right-going eigenvector
        B0, dV, c = (1.0, 0.0, 0.0), [0, 0, 1.0, 0, 0, -1.0, 0, 0, 0], 1.0
    elif kind == "sound":  # B = 0: right-going sound wave
        a = math.sqrt(gam * p0 / rho0)
        B0, dV, c = (0.0, 0.0, 0.0), [rho0, a, 0, 0, 0, 0, 0, gam * p0, 0], a
    elif kind == "fast":  # B perpendicular to k: fast magnetosonic wave
        b = 0.8
        cf = math.sqrt((gam * p0 + b * b) / rho0)
        B0, dV, c = (0.0, b, 0.0), [rho0, cf, 0, 0, 0, b, 0, gam * p0, 0], cf
    pb = Problem("wave", (n, 1, 1), limiter=limiter, cfl=0.8, t_end=1.0 / c,
                 params={"ic": "linear_wave", "rho0": rho0, "p0": p0, "B0": B0,
                         "dV": dV, "amp": 1e-6})
    return pb


@pytest.mark.parametrize("kind", ["alfven", "sound", "fast"])
def test_linear_wave_second_order_mc(kind):
    errs = []
    ns = [64, 128, 256]
    for n in ns:
        pb = _wave_problem(kind, n, orc.LIM_MC)
        g = grid_of(pb)
        V0 = pb.prim()
        r = orc.run(orc.prim_to_cons(V0, pb.gamma), g, 100000, t_end=pb.t_end)
        assert r.t == pytest.approx(pb.t_end, rel=1e-14)
        V1, _ = orc.cons_to_prim(r.U, g)
        var = VY if kind == "alfven" else VX
        errs.append(np.mean(np.abs(V1[var] - V0[var])) / 1e-6)
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    # MC clips the extrema of the sine, so the order approaches 2 from below
    assert orders[-1] >= 1.8 and min(orders) >= 1.6, (errs, orders)
    assert errs[-1] < 0.01


# ------------------------------------------------------------------- JVP --
def test_dual_jvp_matches_central_differences():
    pb = Problem("random_smooth", (8, 7, 1), seed=10)
    g = grid_of(pb)
    U0 = cons_of(pb)
    r = orc.run(U0, g, 3)
    rng = np.random.default_rng(1)
    dU = rng.standard_normal(U0.shape) * np.abs(U0).mean(axis=(1, 2, 3), keepdims=True)
    _, jvp = orc.run_jvp(U0, dU, g, r.dts, r.chs)
    eps = 1e-6
    up = orc.run(U0 + eps * dU, g, 3, dts=r.dts, chs=r.chs).U
    dn = orc.run(U0 - eps * dU, g, 3, dts=r.dts, chs=r.chs).U
    fd = (up - dn) / (2 * eps)
    assert np.max(np.abs(fd - jvp)) <= 1e-6 * np.max(np.abs(jvp))


# ------------------------------------------- one step from pinned pieces --
def _rhs_from_pieces(W, g, ch):
    """L(W) of Section 3.2's five steps, composed in numpy from the oracle's
    separately pinned pieces: ghost fill (= numpy.pad), cons->prim, the
    limited slope (hand values) with the flat fallback for a non-positive
    face density or pressure, and the GLM + HLLD interface flux; the right-
    hand side -(F_{i+1/2} - F_{i-1/2}) / dx_d summed over active d in x, y, z
    order (the oracle's order, so the sums round alike)."""
    Vp, _ = orc.cons_to_prim(orc.fill_ghosts(W, g), g)
    gh = [g.ghost if n > 1 else 0 for n in g.n]
    nx, ny, nz = g.n
    L = np.zeros((9, nz, ny, nx))
    for d in range(3):
        n = g.n[d]
        if n <= 1:
            continue
        ax = 3 - d  # array axes (var, z, y, x)

        def cells(off):  # cells -1 .. n along d shifted by off; interior across
            idx = [slice(None)] * 4
            for a in range(3):
                lo = gh[a] + (off - 1 if a == d else 0)
                idx[3 - a] = slice(lo, lo + g.n[a] + (2 if a == d else 0))
            return Vp[tuple(idx)]

        v0 = cells(0)
        if g.limiter == orc.LIM_WENOZ:  # WENO-Z values at the cell's two faces
            st = np.stack([cells(o) for o in (-2, -1, 0, 1, 2)]).reshape(5, -1)
            plus = orc.wenoz_face(st).reshape(v0.shape)
            minus = orc.wenoz_face(st[::-1]).reshape(v0.shape)
        else:
            sig = orc.limited_slope(v0 - cells(-1), cells(1) - v0, g.limiter)
            plus, minus = v0 + 0.5 * sig, v0 - 0.5 * sig
        bad = (plus[RHO] <= 0) | (minus[RHO] <= 0) | (plus[PRS] <= 0) | (minus[PRS] <= 0)
        plus, minus = np.where(bad, v0, plus), np.where(bad, v0, minus)
        # face f = 0..n between cells f-1 (its + value) and f (its - value)
        VL = np.take(plus, np.arange(0, n + 1), axis=ax)
        VR = np.take(minus, np.arange(1, n + 2), axis=ax)
        F = orc.interface_flux(VL.reshape(9, -1), VR.reshape(9, -1), d, ch,
                               g.gamma).reshape(VL.shape)
        L -= (np.take(F, np.arange(1, n + 1), axis=ax) - np.take(F, np.arange(0, n), axis=ax)) \
            / g.dx[d]
    return L


@pytest.mark.parametrize("pb", [
    Problem("random_smooth", (7, 6, 5), seed=51, bc=(0, 0, 1, 1, 0, 0),
            params={"psi_amp": 1.0}),
    Problem("random_smooth", (9, 8, 1), seed=52, limiter=orc.LIM_MINMOD, bc=(1,) * 6),
    Problem("random_smooth", (8, 7, 6), seed=53, limiter=orc.LIM_WENOZ, rk_order=3,
            bc=(1, 1, 0, 0, 0, 0), params={"psi_amp": 1.0}),
], ids=["3d_mc_mixed_bc", "2d_minmod_outflow", "3d_wenoz_rk3"])
def test_step_rebuilt_from_pinned_pieces(pb):
    """RK2: U1 = U + dt L(U), U^{n+1} = U/2 + (U1 + dt L(U1))/2; SSP-RK3 (Shu
    & Osher): U1 as RK2, U2 = 3U/4 + (U1 + dt L(U1))/4, U^{n+1} = U/3 +
    2(U2 + dt L(U2))/3; then psi times exp(-alpha c_h dt / dh_min) (the
    damping).  With L rebuilt from the pinned pieces, each stage equals
    orc.stage and the step equals one orc.run step, bit for bit (same
    operations in the same order; the oracle is built without FMA
    contraction)."""
    g = grid_of(pb)
    U = cons_of(pb)
    dt, ch = orc.cfl_dt(U, g)
    if g.rk_order == 3:
        coeffs = [(0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0)]
    else:
        coeffs = [(0.0, 1.0), (0.5, 0.5)]
    W = U
    for k, (a_n, a_w) in enumerate(coeffs):
        s1 = W + dt * _rhs_from_pieces(W, g, ch)
        nxt = s1 if k == 0 else a_n * U + a_w * s1
        ref, cnt = orc.stage(W, g, dt, ch, k + 1, Un=None if k == 0 else U)
        assert cnt == (0, 0)
        np.testing.assert_array_equal(ref, nxt)
        W = nxt
    dh = min(g.dx[d] for d in range(3) if g.n[d] > 1)
    W = W.copy()
    W[PSI] *= math.exp(-g.glm_alpha * ch * dt / dh)
    r = orc.run(U, g, 1, dts=[dt], chs=[ch])
    np.testing.assert_array_equal(r.U, W)
