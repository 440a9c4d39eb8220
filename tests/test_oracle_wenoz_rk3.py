"""Pins of the oracle's WENO-Z reconstruction and SSP-RK3 stages (the paper's
own scheme, Section 4.2) against facts independent of the oracle: exactness
for quadratics from exact cell averages, fifth-order convergence of the face
value on smooth data, upwind selection across a discontinuity, the linear
(B_x, psi) subsystem against an independently written upwind SSP-RK3, and
conservation, symmetry and convergence of the full scheme."""
import math

import numpy as np
import pytest

import oracle as orc
from paper_2510_24175_gb300 import inputs
from paper_2510_24175_gb300.inputs import Problem

RHO, VX, VY, VZ, BX, BY, BZ, PRS, PSI = range(9)


def grid_of(pb):
    return orc.Grid(n=pb.n, dx=pb.dx, gamma=pb.gamma, glm_alpha=pb.glm_alpha,
                    rho_floor=pb.rho_floor, p_floor=pb.p_floor, limiter=pb.limiter, bc=pb.bc,
                    cfl=pb.cfl, rk_order=pb.rk_order)


def test_wenoz_exact_for_quadratic_cell_averages():
    rng = np.random.default_rng(1)
    n = 2000
    a, b, c = rng.normal(size=(3, n))
    h = np.exp(rng.uniform(-3, 0, n))
    x0 = rng.normal(size=n)

    def avg(xl):  # exact cell average of a + b x + c x^2 over [xl, xl + h]
        xr = xl + h
        return a + b * (xl + xr) / 2 + c * (xr ** 3 - xl ** 3) / (3 * h)

    f = np.stack([avg(x0 + (j - 2) * h) for j in range(5)])  # cells i-2..i+2, cell i = [x0, x0+h]
    xf = x0 + h
    exact = a + b * xf + c * xf ** 2
    got = orc.wenoz_face(f)
    scale = np.abs(a) + np.abs(b * xf) + np.abs(c * xf ** 2)
    assert np.max(np.abs(got - exact) / scale) < 1e-12


def test_wenoz_fifth_order_on_smooth_data():
    errs = []
    for n in (20, 40, 80):
        h = 1.0 / n
        xl = np.arange(n) * h

        def avg(x):  # exact average of sin(2 pi x) over [x, x+h]
            return (np.cos(2 * math.pi * x) - np.cos(2 * math.pi * (x + h))) / (2 * math.pi * h)

        f = np.stack([avg(xl + (j - 2) * h) for j in range(5)])
        errs.append(np.max(np.abs(orc.wenoz_face(f) - np.sin(2 * math.pi * (xl + h)))))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 4.5, (errs, orders)


def test_wenoz_picks_the_smooth_stencil_across_a_jump():
    f = np.array([[0.0], [0.0], [1.0], [1.0], [1.0]])  # jump between cells i-1 and i
    assert abs(orc.wenoz_face(f)[0] - 1.0) < 1e-30
    f = np.array([[0.0], [0.0], [0.0], [1.0], [1.0]])  # jump between cells i and i+1
    assert abs(orc.wenoz_face(f)[0]) < 1e-30
    # uniform data: exact, ideal weights
    assert orc.wenoz_face(np.full((5, 1), 3.5))[0] == 3.5


def test_rk3_glm_subsystem_matches_linear_upwind():
    """First-order reconstruction + SSP-RK3: (B_x, psi) evolve as the upwind
    scheme for w+- = psi +- ch B_x with the Shu-Osher stages
    u1 = u + dt L(u), u2 = 3/4 u + 1/4 (u1 + dt L(u1)),
    u' = 1/3 u + 2/3 (u2 + dt L(u2)), then psi damping."""
    n = 32
    x = (np.arange(n) + 0.5) / n
    pb = Problem("uniform", (n, 1, 1), limiter=orc.LIM_FLAT, glm_alpha=0.3, rk_order=3,
                 params={"V0": [1.0, 0.1, 0.0, 0.0, 0.0, 0.2, 0.0, 1.0, 0.0]})
    V = pb.prim()
    V[BX, 0, 0, :] = 0.1 * np.sin(2 * np.pi * x)
    V[PSI, 0, 0, :] = 0.05 * np.cos(4 * np.pi * x)
    g = grid_of(pb)
    ch, dt, dx = 2.0, 0.01, 1.0 / n
    r = orc.run(orc.prim_to_cons(V, pb.gamma), g, 3, dts=[dt] * 3, chs=[ch] * 3)
    b, psi = V[BX, 0, 0].copy(), V[PSI, 0, 0].copy()

    def L(wp, wm):
        return (-ch * (wp - np.roll(wp, 1)) / dx, ch * (np.roll(wm, -1) - wm) / dx)

    for _ in range(3):
        wp, wm = psi + ch * b, psi - ch * b
        a1, b1 = L(wp, wm)
        p1, m1 = wp + dt * a1, wm + dt * b1
        a2, b2 = L(p1, m1)
        p2, m2 = 0.75 * wp + 0.25 * (p1 + dt * a2), 0.75 * wm + 0.25 * (m1 + dt * b2)
        a3, b3 = L(p2, m2)
        wp = wp / 3 + 2 / 3 * (p2 + dt * a3)
        wm = wm / 3 + 2 / 3 * (m2 + dt * b3)
        b = (wp - wm) / (2 * ch)
        psi = (wp + wm) / 2 * math.exp(-0.3 * ch * dt / dx)
    np.testing.assert_allclose(r.U[BX, 0, 0], b, rtol=0, atol=1e-14)
    np.testing.assert_allclose(r.U[PSI, 0, 0], psi, rtol=0, atol=1e-14)


def test_wenoz_rk3_periodic_conservation_and_point_symmetry():
    pb = Problem("random_smooth", (12, 10, 8), seed=5, limiter=orc.LIM_WENOZ, rk_order=3)
    g = grid_of(pb)
    U0 = orc.prim_to_cons(pb.prim(), pb.gamma)
    s0 = orc.conserved_sums(U0, g)
    r = orc.run(U0, g, 5)
    s1 = orc.conserved_sums(r.U, g)
    scale = np.maximum(np.abs(s0), orc.conserved_sums(np.abs(U0), g))
    assert np.all(np.abs(s1 - s0) <= 1e-13 * scale)
    ot = inputs.orszag_tang_3d(16, steps=3)
    ot.limiter, ot.rk_order = orc.LIM_WENOZ, 3
    U = orc.run(orc.prim_to_cons(ot.prim(), ot.gamma), grid_of(ot), 3).U
    sym = np.array([1, -1, -1, -1, -1, -1, -1, 1, 1.0])[:, None, None, None]
    sc = np.max(np.abs(U), axis=(1, 2, 3), keepdims=True)
    sc = np.maximum(sc, 1e-3 * sc[RHO])
    assert np.max(np.abs(U - sym * U[:, ::-1, ::-1, ::-1]) / sc) < 1e-12


def test_wenoz_rk3_translation_invariance_and_uniform_state():
    pb = Problem("random_smooth", (8, 6, 5), seed=7, limiter=orc.LIM_WENOZ, rk_order=3)
    g = grid_of(pb)
    U0 = orc.prim_to_cons(pb.prim(), pb.gamma)
    a = orc.run(U0, g, 2).U
    b = orc.run(np.roll(U0, (1, 2, 3), axis=(1, 2, 3)), g, 2).U
    np.testing.assert_array_equal(np.roll(a, (1, 2, 3), axis=(1, 2, 3)), b)
    pu = Problem("uniform", (6, 5, 4), limiter=orc.LIM_WENOZ, rk_order=3, bc=(1,) * 6,
                 params={"V0": [1.3, 0.2, -0.4, 0.1, 0.5, -0.3, 0.7, 0.9, 0.0]})
    Uu = orc.prim_to_cons(pu.prim(), pu.gamma)
    np.testing.assert_allclose(orc.run(Uu, grid_of(pu), 2).U, Uu, rtol=2e-15, atol=2e-15)


@pytest.mark.parametrize("kind", ["alfven", "sound"])
def test_wenoz_rk3_linear_wave_third_order(kind):
    """With CFL fixed, dt ~ dx and the RK3 time error sets the order (3)."""
    rho0, p0, gam = 1.0, 1.0, 5.0 / 3.0
    if kind == "alfven":
        B0, dV, c = (1.0, 0.0, 0.0), [0, 0, 1.0, 0, 0, -1.0, 0, 0, 0], 1.0
    else:
        a = math.sqrt(gam * p0 / rho0)
        B0, dV, c = (0.0, 0.0, 0.0), [rho0, a, 0, 0, 0, 0, 0, gam * p0, 0], a
    errs = []
    for n in (16, 32, 64):
        pb = Problem("wave", (n, 1, 1), limiter=orc.LIM_WENOZ, rk_order=3, t_end=1.0 / c,
                     params={"ic": "linear_wave", "rho0": rho0, "p0": p0, "B0": B0,
                             "dV": dV, "amp": 1e-6})
        V0 = pb.prim()
        r = orc.run(orc.prim_to_cons(V0, pb.gamma), grid_of(pb), 100000, t_end=pb.t_end)
        V1, _ = orc.cons_to_prim(r.U, grid_of(pb))
        var = VY if kind == "alfven" else VX
        errs.append(np.mean(np.abs(V1[var] - V0[var])) / 1e-6)
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) >= 2.8, (errs, orders)


def test_wenoz_dual_jvp_matches_central_differences():
    pb = Problem("random_smooth", (8, 7, 1), seed=10, limiter=orc.LIM_WENOZ, rk_order=3)
    g = grid_of(pb)
    U0 = orc.prim_to_cons(pb.prim(), pb.gamma)
    r = orc.run(U0, g, 2)
    rng = np.random.default_rng(1)
    dU = rng.standard_normal(U0.shape) * np.abs(U0).mean(axis=(1, 2, 3), keepdims=True)
    _, jvp = orc.run_jvp(U0, dU, g, r.dts, r.chs)
    eps = 1e-6
    up = orc.run(U0 + eps * dU, g, 2, dts=r.dts, chs=r.chs).U
    dn = orc.run(U0 - eps * dU, g, 2, dts=r.dts, chs=r.chs).U
    assert np.max(np.abs((up - dn) / (2 * eps) - jvp)) <= 1e-6 * np.max(np.abs(jvp))


def _beta_and_face_from_definition(f, h=1.0):
    """For stencil k (cells i-2+k .. i+k) fit the quadratic whose cell averages
    match f, then beta_k = sum_{l=1,2} h^(2l-1) int_cell_i (p^(l))^2 dx and
    q_k = p(x_{i+1/2}) (Jiang & Shu 1996, their definition of the smoothness
    indicators).  Cell i = [0, h]."""
    betas, qs = [], []
    for k in range(3):
        cells = [(j - 2 + k) for j in range(3)]  # offsets of the stencil cells
        A = []
        for c in cells:  # average of 1, x, x^2 over [c h, (c+1) h]
            xl, xr = c * h, (c + 1) * h
            A.append([1.0, (xl + xr) / 2, (xr ** 3 - xl ** 3) / (3 * h)])
        a0, a1, a2 = np.linalg.solve(np.array(A), f[k:k + 3])
        # p' = a1 + 2 a2 x, p'' = 2 a2 on [0, h]
        int_d1 = a1 ** 2 * h + 2 * a1 * a2 * h ** 2 + 4 * a2 ** 2 * h ** 3 / 3
        int_d2 = 4 * a2 ** 2 * h
        betas.append(h * int_d1 + h ** 3 * int_d2)
        qs.append(a0 + a1 * h + a2 * h * h)
    return np.array(betas), np.array(qs)


def test_wenoz_weights_from_the_smoothness_indicator_definition():
    """WENO-Z (Borges et al. 2008, exponent 1): alpha_k = d_k (1 + tau5 /
    (beta_k + eps)), tau5 = |beta_0 - beta_2|, d = (1/10, 6/10, 3/10); with
    beta_k and q_k derived independently above, on random rough data."""
    rng = np.random.default_rng(4)
    F = rng.normal(size=(5, 200)) * np.exp(rng.uniform(-2, 2, size=(1, 200)))
    got = orc.wenoz_face(F)
    d = np.array([0.1, 0.6, 0.3])
    for i in range(F.shape[1]):
        beta, q = _beta_and_face_from_definition(F[:, i])
        tau = abs(beta[0] - beta[2])
        alpha = d * (1.0 + tau / (beta + 1e-40))
        ref = float(np.sum(alpha * q) / np.sum(alpha))
        assert abs(got[i] - ref) <= 1e-11 * (np.max(np.abs(F[:, i])) + 1e-300), i
