"""Pins of the oracle's interface flux (GLM step + HLLD), fast speed and
limiters against facts that do not come from the oracle itself:
textbook MHD fluxes, an independently written HLLC solver (the B = 0 limit of
HLLD), the characteristic solution of the linear (B_n, psi) system, exact
resolution of isolated contact and rotational discontinuities (a stated
property of HLLD, Miyoshi & Kusano 2005), reflection and rotation symmetry,
eigenvalues of the 1-D MHD Jacobian, and hand-computed limiter values.
"""
import math

import numpy as np
import pytest

import oracle as orc
from paper_2510_24175_gb300 import inputs

RHO, VX, VY, VZ, BX, BY, BZ, PRS, PSI = range(9)
GAMMA = 5.0 / 3.0


def textbook_flux(V, d, ch, gamma):
    """Ideal-MHD flux along axis d (B treated with 4 pi absorbed) plus the
    GLM pair F[B_n] = psi, F[psi] = ch^2 B_n, for VL = VR (GLM is the identity)."""
    rho, p = V[RHO], V[PRS]
    v = V[VX:VZ + 1]
    B = V[BX:BZ + 1]
    v2 = np.sum(v * v, axis=0)
    b2 = np.sum(B * B, axis=0)
    E = p / (gamma - 1) + 0.5 * rho * v2 + 0.5 * b2
    pt = p + 0.5 * b2
    vn, bn = v[d], B[d]
    F = np.empty_like(V)
    F[RHO] = rho * vn
    for a in range(3):
        F[VX + a] = rho * v[a] * vn - B[a] * bn + (pt if a == d else 0.0)
        F[BX + a] = vn * B[a] - v[a] * bn
    F[BX + d] = V[PSI]
    F[PRS] = (E + pt) * vn - bn * np.sum(v * B, axis=0)
    F[PSI] = ch * ch * bn
    return F


def test_consistency_equal_states():
    """F(V, V) = F(V) for random states in all three directions."""
    VL, _ = inputs.random_face_states(2000, seed=11)
    for d in range(3):
        F = orc.interface_flux(VL, VL, d, ch=1.7, gamma=GAMMA)
        ref = textbook_flux(VL, d, 1.7, GAMMA)
        np.testing.assert_allclose(F, ref, rtol=1e-12, atol=1e-12)


def _supersonic(sign, count=500):
    VL, VR = inputs.random_face_states(count, seed=12)
    for V in (VL, VR):
        V[VX] = sign * (50.0 + np.abs(V[VX]))
        V[PSI] = 0.0
    VR[BX] = VL[BX]  # continuous normal field: GLM is the identity
    return VL, VR


def test_supersonic_upwinding():
    VL, VR = _supersonic(+1)
    F = orc.interface_flux(VL, VR, 0, ch=1.0, gamma=GAMMA)
    np.testing.assert_allclose(F, textbook_flux(VL, 0, 1.0, GAMMA), rtol=1e-13, atol=1e-13)
    VL, VR = _supersonic(-1)
    F = orc.interface_flux(VL, VR, 0, ch=1.0, gamma=GAMMA)
    np.testing.assert_allclose(F, textbook_flux(VR, 0, 1.0, GAMMA), rtol=1e-13, atol=1e-13)


def hllc_toro(VL, VR, gamma):
    """HLLC for the Euler equations (Toro, Riemann Solvers and Numerical
    Methods, 3rd ed., Sect. 10.4), with wave speeds min(u)-max(a), max(u)+max(a).
    Returns (rho, mx, my, mz, E) fluxes along x."""
    out = np.empty((5, VL.shape[1]))
    for f in range(VL.shape[1]):
        def prim(V):
            rho, u, v, w, p = V[RHO, f], V[VX, f], V[VY, f], V[VZ, f], V[PRS, f]
            E = p / (gamma - 1) + 0.5 * rho * (u * u + v * v + w * w)
            U = np.array([rho, rho * u, rho * v, rho * w, E])
            F = np.array([rho * u, rho * u * u + p, rho * u * v, rho * u * w, u * (E + p)])
            return rho, u, v, w, p, E, U, F, math.sqrt(gamma * p / rho)
        rl, ul, vl, wl, pl, El, Ul, Fl, al = prim(VL)
        rr, ur, vr, wr, pr, Er, Ur, Fr, ar = prim(VR)
        sl = min(ul, ur) - max(al, ar)
        sr = max(ul, ur) + max(al, ar)
        if sl > 0:
            out[:, f] = Fl
            continue
        if sr < 0:
            out[:, f] = Fr
            continue
        ss = (pr - pl + rl * ul * (sl - ul) - rr * ur * (sr - ur)) / (rl * (sl - ul) - rr * (sr - ur))

        def star(r, u, v, w, p, E, s):
            fac = r * (s - u) / (s - ss)
            return fac * np.array([1.0, ss, v, w,
                                   E / r + (ss - u) * (ss + p / (r * (s - u)))])
        if ss >= 0:
            out[:, f] = Fl + sl * (star(rl, ul, vl, wl, pl, El, sl) - Ul)
        else:
            out[:, f] = Fr + sr * (star(rr, ur, vr, wr, pr, Er, sr) - Ur)
    return out


def test_b0_limit_is_hllc():
    VL, VR = inputs.random_face_states(400, seed=13, degenerate="b0")
    F = orc.interface_flux(VL, VR, 0, ch=1.0, gamma=GAMMA)
    ref = hllc_toro(VL, VR, GAMMA)
    np.testing.assert_allclose(F[[RHO, VX, VY, VZ, PRS]], ref, rtol=1e-11, atol=1e-12)
    # magnetic fluxes vanish with B = 0 and psi = 0
    np.testing.assert_array_equal(F[BX:BZ + 1], 0.0)
    np.testing.assert_array_equal(F[PSI], 0.0)


def test_glm_pair_is_characteristic_upwind():
    """(F[B_n], F[psi]) is the exact upwind flux of the linear system
    B_t + psi_x = 0, psi_t + ch^2 B_x = 0: w+ = psi + ch B (speed +ch) taken
    from the left, w- = psi - ch B (speed -ch) from the right."""
    VL, VR = inputs.random_face_states(1000, seed=14)
    ch = 2.3
    for d in range(3):
        F = orc.interface_flux(VL, VR, d, ch=ch, gamma=GAMMA)
        wp = VL[PSI] + ch * VL[BX + d]
        wm = VR[PSI] - ch * VR[BX + d]
        bn = (wp - wm) / (2 * ch)
        psi = (wp + wm) / 2
        np.testing.assert_allclose(F[BX + d], psi, rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(F[PSI], ch * ch * bn, rtol=1e-13, atol=1e-13)


def _pair_from(VLcols, VRcols):
    VL = np.array(VLcols, dtype=np.float64).reshape(9, -1)
    VR = np.array(VRcols, dtype=np.float64).reshape(9, -1)
    return VL, VR


@pytest.mark.parametrize("u", [0.0, 0.4, -0.3])
def test_isolated_contact_exact(u):
    """A contact (density jump only, u, v, w, p, B continuous) is resolved
    exactly: the flux is the physical flux of the upwind state."""
    VL, VR = _pair_from([1.0, u, 0.2, -0.1, 0.7, 0.3, -0.2, 1.0, 0.0],
                        [0.3, u, 0.2, -0.1, 0.7, 0.3, -0.2, 1.0, 0.0])
    F = orc.interface_flux(VL, VR, 0, ch=1.0, gamma=GAMMA)
    up = VL if u >= 0 else VR
    np.testing.assert_allclose(F, textbook_flux(up, 0, 1.0, GAMMA), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("direction", [+1, -1])
def test_isolated_rotational_discontinuity_exact(direction):
    """A rotational (Alfven) discontinuity moving at +-Bn/sqrt(rho) in a static
    fluid is resolved exactly: the flux at the interface is the physical flux
    of the state on the side the wave is moving away from."""
    rho, p, bn = 1.3, 0.8, 0.9
    ca = bn / math.sqrt(rho)
    ang_l, ang_r = 0.3, 1.9
    bt = 0.6
    BL = np.array([bt * math.cos(ang_l), bt * math.sin(ang_l)])
    BR = np.array([bt * math.cos(ang_r), bt * math.sin(ang_r)])
    # jump condition across an Alfven wave of speed s = direction * ca:
    # [v_t] = -[B_t] bn / (rho s)
    s = direction * ca
    vL = np.array([0.05, -0.02])
    vR = vL - (BR - BL) * bn / (rho * s)
    VL, VR = _pair_from([rho, 0.0, vL[0], vL[1], bn, BL[0], BL[1], p, 0.0],
                        [rho, 0.0, vR[0], vR[1], bn, BR[0], BR[1], p, 0.0])
    F = orc.interface_flux(VL, VR, 0, ch=1.0, gamma=GAMMA)
    up = VL if direction > 0 else VR
    np.testing.assert_allclose(F, textbook_flux(up, 0, 1.0, GAMMA), rtol=1e-12, atol=1e-13)


def _perm_state(V, d):
    """Rotate axes so that axis d becomes x: (x, y, z) <- (d, d+1, d+2)."""
    W = V.copy()
    for a in range(3):
        W[VX + a] = V[VX + (d + a) % 3]
        W[BX + a] = V[BX + (d + a) % 3]
    return W


def test_rotation_invariance():
    VL, VR = inputs.random_face_states(1000, seed=15)
    for d in range(3):
        Fd = orc.interface_flux(VL, VR, d, ch=1.3, gamma=GAMMA)
        Fx_rot = orc.interface_flux(_perm_state(VL, d), _perm_state(VR, d), 0, ch=1.3,
                                    gamma=GAMMA)
        # equal up to the summation order of |B|^2 and |v|^2
        np.testing.assert_allclose(_perm_state(Fd, d), Fx_rot, rtol=1e-11, atol=1e-13)


def test_reflection_symmetry():
    """x -> -x: (u, Bx) change sign (B treated as a polar vector, which the
    ideal-MHD system permits because it is invariant under B -> -B).  Then
    F(M VR, M VL) = -M F(VL, VR) with M = diag(1,-1,1,1,-1,1,1,1,1)."""
    VL, VR = inputs.random_face_states(1000, seed=16)
    M = np.array([1, -1, 1, 1, -1, 1, 1, 1, 1], dtype=np.float64)[:, None]
    F = orc.interface_flux(VL, VR, 0, ch=1.1, gamma=GAMMA)
    Fm = orc.interface_flux(M * VR, M * VL, 0, ch=1.1, gamma=GAMMA)
    np.testing.assert_allclose(Fm, -M * F, rtol=1e-12, atol=1e-13)


def mhd_jacobian_eigs(V, gamma):
    """Eigenvalues of the 1-D ideal-MHD system in primitive form
    q = (rho, u, v, w, By, Bz, p) along x with constant Bx."""
    rho, u, v, w = V[RHO], V[VX], V[VY], V[VZ]
    bx, by, bz, p = V[BX], V[BY], V[BZ], V[PRS]
    A = np.zeros((7, 7))
    A[0] = [u, rho, 0, 0, 0, 0, 0]
    A[1] = [0, u, 0, 0, by / rho, bz / rho, 1 / rho]
    A[2] = [0, 0, u, 0, -bx / rho, 0, 0]
    A[3] = [0, 0, 0, u, 0, -bx / rho, 0]
    A[4] = [0, by, -bx, 0, u, 0, 0]
    A[5] = [0, bz, 0, -bx, 0, u, 0]
    A[6] = [0, gamma * p, 0, 0, 0, 0, u]
    return np.linalg.eigvals(A).real


def test_fast_speed_matches_jacobian_eigenvalues():
    VL, _ = inputs.random_face_states(200, seed=17)
    cf = orc.fast_speed(VL, 0, GAMMA)
    for f in range(VL.shape[1]):
        lam = mhd_jacobian_eigs(VL[:, f], GAMMA)
        assert abs((lam.max() - VL[VX, f]) - cf[f]) <= 1e-9 * cf[f]


def test_fast_speed_special_cases():
    V = np.zeros((9, 3))
    V[RHO] = 2.0
    V[PRS] = 1.5
    V[BX:BZ + 1, 1] = [0.0, 0.8, 0.6]   # B perpendicular to x
    V[BX, 2] = 3.0                       # B along x, Alfven faster than sound
    cf = orc.fast_speed(V, 0, GAMMA)
    a2 = GAMMA * 1.5 / 2.0
    np.testing.assert_allclose(cf[0], math.sqrt(a2), rtol=1e-15)
    np.testing.assert_allclose(cf[1], math.sqrt(a2 + 1.0 / 2.0), rtol=1e-15)
    np.testing.assert_allclose(cf[2], 3.0 / math.sqrt(2.0), rtol=1e-15)


@pytest.mark.parametrize("lim,dm,dp,expect", [
    (orc.LIM_MINMOD, 1.0, 2.0, 1.0), (orc.LIM_MINMOD, -3.0, -1.0, -1.0),
    (orc.LIM_MINMOD, 1.0, -1.0, 0.0), (orc.LIM_MINMOD, 0.0, 5.0, 0.0),
    (orc.LIM_MC, 1.0, 2.0, 1.5), (orc.LIM_MC, 1.0, 5.0, 2.0),
    (orc.LIM_MC, -1.0, -1.2, -1.1), (orc.LIM_MC, -4.0, -0.5, -1.0),
    (orc.LIM_MC, 2.0, -1.0, 0.0), (orc.LIM_FLAT, 1.0, 1.0, 0.0),
])
def test_limiter_values(lim, dm, dp, expect):
    out = orc.limited_slope(np.array([dm]), np.array([dp]), lim)
    assert out[0] == expect


def test_limiters_reproduce_linear_data():
    d = np.linspace(-3, 3, 13)
    for lim in (orc.LIM_MINMOD, orc.LIM_MC):
        np.testing.assert_array_equal(orc.limited_slope(d, d, lim), d)


def test_flux_continuous_as_waves_cross_the_interface():
    """Adding a uniform normal velocity U to both states sweeps every wave of
    the HLLD fan across the interface.  The HLLD states are built so that
    the fluxes of neighbouring fan regions agree where a wave speed is zero
    (Rankine-Hugoniot across each wave, continuity across S_M), so the flux is
    a continuous function of U: no jump larger than a Lipschitz bound."""
    VL0, VR0 = inputs.random_face_states(12, seed=22)
    Us = np.linspace(-6.0, 6.0, 40001)
    dU = Us[1] - Us[0]
    for f in range(VL0.shape[1]):
        VL = np.repeat(VL0[:, f:f + 1], Us.size, axis=1)
        VR = np.repeat(VR0[:, f:f + 1], Us.size, axis=1)
        VR[BX] = VL[BX]          # GLM identity: keep the normal field continuous
        VL[PSI] = VR[PSI] = 0.0
        VR[RHO] *= 3.0           # unequal star densities on the two sides
        VL[VX] += Us
        VR[VX] += Us
        F = orc.interface_flux(VL, VR, 0, ch=1.0, gamma=GAMMA)
        jumps = np.abs(np.diff(F, axis=1))
        slope = np.median(jumps, axis=1, keepdims=True) / dU + 1.0
        assert np.all(jumps <= 200.0 * slope * dU), f
