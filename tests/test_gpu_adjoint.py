"""Discrete adjoint (mhd_adjoint_step, MHDRollout) against the oracle's exact
forward-mode derivative (dual numbers) and against central finite
differences.  dt and c_h are frozen (recorded) in every comparison.

Tolerances: step adjoint vs oracle JVP 1e-11 relative (dot-product identity
and full Jacobian); rollout gradient vs oracle JVP 1e-9 relative; rollout
gradient vs central differences 1e-6 relative to the gradient scale
||grad J|| ||d||.  The discrete map is only piecewise smooth (limiter
extrema and switches, wave-speed min/max), so central differences carry kink
errors at large epsilon and round-off at small epsilon: on this objective
the oracle's own exact JVP and its own central differences differ by 2e-6 to
2e-5 relative to a random direction's derivative, which is ~sqrt(n) times
smaller than ||grad J|| ||d||; the best epsilon of a 1e-3 .. 1e-6 sweep is
taken.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2510_24175_gb300 import inputs
from paper_2510_24175_gb300.inputs import Problem
from parity_util import grid_of

pytestmark = pytest.mark.gpu


def _solver(pb):
    from paper_2510_24175_gb300.adjoint import rollout_solver
    return rollout_solver(pb)


def _gpu_adjoint(s, U, lam, dt, ch):
    import torch
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    Ld = torch.from_numpy(np.ascontiguousarray(lam)).cuda()
    out = torch.empty_like(Ld)
    s.adjoint_step(Ud, Ld, out, dt, ch)
    return out.cpu().numpy()


CASES = [
    Problem("random_smooth", (12, 10, 1), seed=31),
    Problem("random_smooth", (9, 7, 5), seed=32, limiter=orc.LIM_MINMOD, bc=(1,) * 6),
    Problem("random_smooth", (10, 6, 4), seed=33, bc=(0, 0, 1, 1, 0, 0),
            params={"psi_amp": 3.0}),
    Problem("random_smooth", (16, 1, 1), seed=34, limiter=orc.LIM_FLAT, bc=(1,) * 6),
]


@pytest.mark.parametrize("pb", CASES, ids=["2d_mc", "3d_minmod_outflow", "3d_mixed_psi",
                                            "1d_flat"])
def test_step_adjoint_dot_product_vs_oracle_jvp(pb):
    g = grid_of(pb)
    U = orc.prim_to_cons(pb.prim(), pb.gamma)
    dt, ch = orc.cfl_dt(U, g)
    s = _solver(pb)
    rng = np.random.default_rng(7)
    for _ in range(3):
        lam = rng.standard_normal(U.shape)
        v = rng.standard_normal(U.shape) * np.abs(U).mean(axis=(1, 2, 3), keepdims=True)
        _, jv = orc.run_jvp(U, v, g, [dt], [ch])
        lhs = float(np.sum(lam * jv))
        adj = _gpu_adjoint(s, U, lam, dt, ch)
        rhs = float(np.sum(adj * v))
        scale = float(np.sum(np.abs(lam * jv)))
        assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs, scale)


@pytest.mark.parametrize("pb", [Problem("random_smooth", (6, 5, 1), seed=41),
                                Problem("random_smooth", (4, 4, 3), seed=42, bc=(1,) * 6,
                                        limiter=orc.LIM_MINMOD)], ids=["2d", "3d_outflow"])
def test_step_adjoint_full_jacobian(pb):
    """J built column by column from the oracle's exact JVP; the GPU adjoint
    must equal J^T lam element by element."""
    g = grid_of(pb)
    U = orc.prim_to_cons(pb.prim(), pb.gamma)
    dt, ch = orc.cfl_dt(U, g)
    n = U.size
    J = np.empty((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        _, col = orc.run_jvp(U, e.reshape(U.shape), g, [dt], [ch])
        J[:, i] = col.ravel()
    s = _solver(pb)
    rng = np.random.default_rng(3)
    for _ in range(2):
        lam = rng.standard_normal(U.shape)
        ref = (J.T @ lam.ravel()).reshape(U.shape)
        got = _gpu_adjoint(s, U, lam, dt, ch)
        scale = np.abs(J).T @ np.abs(lam.ravel())
        err = np.abs(got.ravel() - ref.ravel()) / (scale + 1e-300)
        assert err.max() < 1e-11, err.max()


def kinetic_energy(U, cell_volume: float):
    """The test's objective J = sum over cells of |m|^2 / (2 rho) times the
    cell volume (user-side code: differentiated by torch, not the library)."""
    return 0.5 * ((U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0]).sum() * cell_volume


def prim_to_cons_torch(V, gamma: float):
    """The test's parameterisation of the initial state: primitive ->
    conservative in torch, so that the gradient reaches the velocity
    perturbation (user-side code, not the library's conversion)."""
    import torch
    rho = V[0]
    v2 = V[1] ** 2 + V[2] ** 2 + V[3] ** 2
    b2 = V[4] ** 2 + V[5] ** 2 + V[6] ** 2
    E = V[7] / (gamma - 1.0) + 0.5 * rho * v2 + 0.5 * b2
    return torch.stack([rho, rho * V[1], rho * V[2], rho * V[3], V[4], V[5], V[6], E, V[8]])

def _rollout_grad(pb, dv, nsteps, k):
    """Gradient of J = kinetic energy at t_N w.r.t. the velocity perturbation
    dv (2, nz, ny, nx) through MHDRollout; returns (J, grad, dts, chs, U0)."""
    import torch
    from paper_2510_24175_gb300.adjoint import MHDRollout
    s = _solver(pb)
    V0 = torch.from_numpy(pb.prim()).cuda()
    p = torch.from_numpy(dv).cuda().requires_grad_(True)
    V = V0.clone()
    V = torch.cat([V[:1], V[1:3] + p, V[3:]])
    U0 = prim_to_cons_torch(V, pb.gamma)
    UN = MHDRollout.apply(U0, s, nsteps, k)
    vol = pb.dx[0] * pb.dx[1]
    J = kinetic_energy(UN, vol)
    J.backward()
    return float(J.detach()), p.grad.cpu().numpy(), U0.detach().cpu().numpy(), s


def _J_frozen(pb, dv, dts, chs):
    """J with the recorded dt / c_h sequence (forward only, through the ABI)."""
    import torch
    import paper_2510_24175_gb300 as m
    s = m.MHD(m.Config.from_problem(pb))
    V = pb.prim()
    V[1:3] += dv
    s.set_state(torch.from_numpy(V).cuda(), kind=m.MHD_PRIM)
    for dt, ch in zip(dts, chs):
        s.step(dt, ch)
    U = s.get_state().cpu().numpy()
    return 0.5 * float(np.sum((U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0])) * pb.dx[0] * pb.dx[1]


def _recorded(pb, dv, nsteps):
    import torch
    import paper_2510_24175_gb300 as m
    s = m.MHD(m.Config.from_problem(pb))
    V = pb.prim()
    V[1:3] += dv
    s.set_state(torch.from_numpy(V).cuda(), kind=m.MHD_PRIM)
    dts, chs = [], []
    for _ in range(nsteps):
        s.step()
        info = s.step_info()
        dts.append(info["dt"])
        chs.append(info["ch"])
    return dts, chs


def test_rollout_gradient_vs_central_differences_and_oracle():
    """2-D Orszag-Tang 64^2, 20 RK2 steps, checkpoints every 5 steps; J =
    kinetic energy; gradient w.r.t. a seeded velocity perturbation (rms 1e-3)
    checked on 16 seeded directions by central differences (epsilon sweep,
    frozen dt/c_h) and by the oracle's dual-number JVP."""
    pb = inputs.orszag_tang_2d(64, steps=20)
    dv = inputs.adjoint_perturbation(pb, seed=4)
    J, grad, U0, _ = _rollout_grad(pb, dv, 20, 5)
    dts, chs = _recorded(pb, dv, 20)
    dirs = inputs.random_directions(dv.shape, 16, seed=4) * np.sqrt(dv.size) * 1e-3
    gnorm = float(np.sqrt(np.sum(grad * grad)))
    worst = 0.0
    for d in dirs[:16]:
        ad = float(np.sum(grad * d))
        scale = gnorm * float(np.sqrt(np.sum(d * d)))
        best = np.inf
        for eps in (1e-3, 1e-4, 1e-5, 1e-6):
            fd = (_J_frozen(pb, dv + eps * d, dts, chs) - _J_frozen(pb, dv - eps * d, dts, chs)) / (2 * eps)
            best = min(best, abs(fd - ad) / scale)
        worst = max(worst, best)
    assert worst < 1e-6, worst

    # oracle: exact directional derivative of J through its own recorded run
    g = grid_of(pb)
    V = pb.prim()
    V[1:3] += dv
    Uo = orc.prim_to_cons(V, pb.gamma)
    ref = orc.run(Uo, g, 20)
    UN = ref.U
    vol = pb.dx[0] * pb.dx[1]
    dJ = np.zeros_like(UN)
    m2 = UN[1] ** 2 + UN[2] ** 2 + UN[3] ** 2
    dJ[0] = -0.5 * m2 / UN[0] ** 2 * vol
    dJ[1:4] = UN[1:4] / UN[0] * vol
    for d in dirs[:4]:
        # dU0 for a velocity direction d: dm = rho d, dE = rho v . d
        dU0 = np.zeros_like(Uo)
        dU0[1:3] = V[0] * d
        dU0[7] = V[0] * (V[1] * d[0] + V[2] * d[1])
        _, jv = orc.run_jvp(Uo, dU0, g, ref.dts, ref.chs)
        lhs = float(np.sum(dJ * jv))
        rhs = float(np.sum(grad * d))
        assert abs(lhs - rhs) <= 1e-9 * abs(lhs), (lhs, rhs)


@pytest.mark.parametrize("pb", [CASES[0], CASES[2]], ids=["2d_mc", "3d_mixed_psi"])
def test_adjoint_with_kept_stage1_equals_recomputed(pb):
    """mhd_get_stage1 after a step with explicit dt, c_h returns that step's
    first RK stage (the oracle's stage 1 within 1e-12 relative L1 per
    variable; host and device copies equal), and mhd_adjoint_step_stage1
    with it gives mhd_adjoint_step's result up to the order of the adjoint's
    FP64 atomic accumulation (run to run a few ulp: 1e-13 of the largest
    component).  set_state clears the kept stage; U1 aliasing U^n is
    rejected."""
    import torch
    import paper_2510_24175_gb300 as m
    g = grid_of(pb)
    U = orc.prim_to_cons(pb.prim(), pb.gamma)
    dt, ch = orc.cfl_dt(U, g)
    s = _solver(pb)
    Ud = torch.from_numpy(U).cuda()
    s.set_state(Ud)
    with pytest.raises(m.MHDError) as e:
        s.get_stage1()
    assert e.value.code == m.MHD_ERR_STATE
    s.step(dt, ch)
    U1 = s.get_stage1()
    U1h = np.empty(U.shape)
    s.get_stage1(U1h)
    np.testing.assert_array_equal(U1.cpu().numpy(), U1h)
    ref, _ = orc.stage(U, g, dt, ch, 1)
    for v in range(9):
        scale = max(float(np.abs(ref[v]).sum()), 1e-300)
        assert float(np.abs(U1h[v] - ref[v]).sum()) / scale < 1e-12, v
    rng = np.random.default_rng(11)
    lam = torch.from_numpy(rng.standard_normal(U.shape)).cuda()
    a = torch.empty_like(lam)
    b = torch.empty_like(lam)
    s.adjoint_step(Ud, lam, a, dt, ch)
    s.adjoint_step_stage1(Ud, U1, lam, b, dt, ch)
    ah, bh = a.cpu().numpy(), b.cpu().numpy()
    np.testing.assert_allclose(bh, ah, rtol=1e-13, atol=1e-13 * float(np.abs(ah).max()))
    with pytest.raises(m.MHDError) as e:
        s.adjoint_step_stage1(Ud, Ud, lam, b, dt, ch)
    assert e.value.code == m.MHD_ERR_INVALID
    s.set_state(Ud)
    with pytest.raises(m.MHDError) as e:
        s.get_stage1()
    assert e.value.code == m.MHD_ERR_STATE


@pytest.mark.parametrize("k", [0, 1, 3, 8])
def test_rollout_gradient_independent_of_checkpoint_interval(k):
    """The rollout's gradient does not depend on the checkpoint interval k
    (k = 0: every step's state and first stage kept by the forward pass, no
    recomputation; k = 1: every step recomputes its first stage inside the
    adjoint; larger k: all but a segment's last step use the first stage kept
    by the segment's recomputation): the gradient
    of k = 8 over 8 steps, which recomputes nothing but the last step's first
    stage, up to the order of the adjoint's FP64 atomic accumulation (1e-11
    of the largest component after 8 steps)."""
    pb = inputs.orszag_tang_2d(32, steps=8)
    dv = inputs.adjoint_perturbation(pb, seed=5)
    _, grad_k, _, _ = _rollout_grad(pb, dv, 8, k)
    _, grad_8, _, _ = _rollout_grad(pb, dv, 8, 8)
    np.testing.assert_allclose(grad_k, grad_8, rtol=1e-11,
                               atol=1e-11 * float(np.abs(grad_8).max()))
