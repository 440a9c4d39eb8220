"""Parity checks at the full sizes of the measured workloads, in the launch
configuration bench.py times (same contexts, same kernels):

* turbulent box 512^3, FP32 bulk: one step at sampled cells against the FP64
  oracle (a cell's new value needs only a 9^3 neighbourhood), and the error of
  the 50-step FP32 state against the FP64 GPU path (which holds 1e-12 against
  the oracle at every size the oracle can run);
* the paper's schemes, WENO-Z + SSP-RK3 with GLM or constrained transport,
  Orszag-Tang 256^3 FP64: one step at sampled cells against the oracle; their
  FP32 lines: 8 steps against the FP64 GPU path;
* batched ensemble of 64 seeded boxes (edges 32..128, FP32, 10 steps in one
  persistent graph launch): bitwise equal to per-box plain launches;
* adjoint of 2-D Orszag-Tang 512^2, 200 RK2 steps, checkpoints every 20 steps:
  gradient against central differences on 16 seeded directions.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2510_24175_gb300 import inputs
from parity_util import sampled_one_step

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _run(pb, nsteps, precision, V):
    import torch
    import paper_2510_24175_gb300 as m
    s = m.MHD(m.Config.from_problem(pb, precision=precision))
    s.set_state(torch.from_numpy(V).cuda(), kind=m.MHD_PRIM)
    for _ in range(nsteps):
        s.step()
    info = s.step_info()
    c = s.counters()
    assert c["rho_floor"] == 0 and c["p_floor"] == 0
    return s, info


def test_turbulent_512_fp32_one_step_sampled_against_oracle():
    pb = inputs.turbulent_box(512)
    V = pb.prim()
    s, info = _run(pb, 1, 1, V)
    U = s.get_state().cpu().numpy()
    U0 = orc.prim_to_cons(V, pb.gamma)
    rng = np.random.default_rng(23)
    cells = [tuple(int(v) for v in rng.integers(0, 512, size=3)) for _ in range(12)]
    cells += [(0, 0, 0), (511, 511, 511), (0, 255, 511)]
    ref = sampled_one_step(U0, pb, info["dt"], info["ch"], cells)
    got = np.stack([U[:, k, j, i] for (k, j, i) in cells], axis=1)
    scale = np.maximum(np.abs(U0).reshape(9, -1).max(axis=1), 0.1 * np.abs(U0[0]).max())
    err = (np.abs(got - ref).max(axis=1) / scale)
    assert np.all(err <= 1e-5), err


def test_turbulent_512_fp32_50_steps_against_fp64_gpu():
    pb = inputs.turbulent_box(512, steps=50)
    V = pb.prim()
    s32, i32 = _run(pb, 50, 1, V)
    U32 = s32.get_state().cpu().numpy()
    del s32
    s64, i64 = _run(pb, 50, 0, V)
    U64 = s64.get_state().cpu().numpy()
    del s64
    assert abs(i32["t"] - i64["t"]) <= 1e-5 * i64["t"]
    num = np.abs(U32 - U64).reshape(9, -1).sum(axis=1)
    den = np.abs(U64).reshape(9, -1).sum(axis=1)
    err = num / np.maximum(den, 0.1 * den[0])
    print("turbulent 512^3 x 50 steps, FP32 vs FP64 rel L1 per variable:", err)
    assert np.all(err <= 1e-5), err


@pytest.mark.parametrize("ct", [False, True])
def test_wenoz_rk3_256_one_step_sampled_against_oracle(ct):
    """The paper's own schemes as bench.py times them (WENO-Z + SSP-RK3 with
    GLM cleaning or constrained transport, Orszag-Tang 256^3, FP64): one step
    on the GPU, the oracle's value at sampled cells (a periodic box around each
    cell, large enough that its boundary cannot reach the centre)."""
    import torch
    import paper_2510_24175_gb300 as m
    from parity_util import grid_of
    pb = inputs.orszag_tang_3d(256)
    pb.limiter, pb.rk_order = m.MHD_LIM_WENOZ, 3
    if ct:
        pb.divb = m.MHD_DIVB_CT
    s = m.MHD(m.Config.from_problem(pb))
    s.set_state(torch.from_numpy(pb.prim()).cuda(), kind=m.MHD_PRIM)
    faces = None
    if ct:
        faces = pb.faces()
        s.set_face_field(torch.from_numpy(faces).cuda())
    U0 = s.get_state().cpu().numpy()
    s.step()
    info = s.step_info()
    dt, _ = orc.cfl_dt(U0, grid_of(pb))
    assert abs(info["dt"] - dt) <= 1e-13 * dt
    U1 = s.get_state().cpu().numpy()
    rng = np.random.default_rng(31 + ct)
    cells = [tuple(int(v) for v in rng.integers(0, 256, 3)) for _ in range(4 if ct else 10)]
    cells += [(0, 0, 0), (255, 255, 255), (0, 255, 128)]
    ref = sampled_one_step(U0, pb, info["dt"], info["ch"], cells, faces=faces)
    got = np.stack([U1[:, k, j, i] for (k, j, i) in cells], axis=1)
    scale = np.abs(U0).reshape(9, -1).max(axis=1)[:, None]
    scale = np.maximum(scale, scale[0])  # B_z and psi start at zero
    err = np.max(np.abs(got - ref) / scale)
    assert err < 1e-12, err


@pytest.mark.parametrize("ct", [False, True])
def test_wenoz_rk3_256_fp32_against_fp64_gpu(ct):
    """The FP32 lines of the paper's schemes (WENO-Z + SSP-RK3, GLM or
    constrained transport, Orszag-Tang 256^3): 8 steps in FP32 against the
    FP64 GPU path (pinned to the oracle at this size by the sampled test)."""
    import torch
    import paper_2510_24175_gb300 as m
    pb = inputs.orszag_tang_3d(256)
    pb.limiter, pb.rk_order = m.MHD_LIM_WENOZ, 3
    if ct:
        pb.divb = m.MHD_DIVB_CT
    res = {}
    for prec in (m.MHD_FP32, m.MHD_FP64):
        s = m.MHD(m.Config.from_problem(pb, precision=prec))
        s.set_state(torch.from_numpy(pb.prim()).cuda(), kind=m.MHD_PRIM)
        if ct:
            s.set_face_field(torch.from_numpy(pb.faces()).cuda())
        for _ in range(8):
            s.step()
        res[prec] = (s.get_state().cpu().numpy(), s.step_info())
        c = s.counters()
        assert c["rho_floor"] == 0 and c["p_floor"] == 0
        del s
    (U32, i32), (U64, i64) = res[m.MHD_FP32], res[m.MHD_FP64]
    assert abs(i32["t"] - i64["t"]) <= 1e-5 * i64["t"]
    num = np.abs(U32 - U64).reshape(9, -1).sum(axis=1)
    den = np.abs(U64).reshape(9, -1).sum(axis=1)
    err = num / np.maximum(den, 0.1 * den[0])
    print("WENO-Z + SSP-RK3", "CT" if ct else "GLM", "256^3 x 8 steps, FP32 vs FP64:", err)
    assert np.all(err <= 1e-5), err


def test_ensemble_64_boxes_bitwise_equal_to_plain_launches():
    import torch
    import paper_2510_24175_gb300 as m
    sizes, b0s = inputs.ensemble_sizes(64, seed=5)
    pbs = []
    for n, b0 in zip(sizes, b0s):
        q = inputs.orszag_tang_3d(n)
        q.params = {"B0": b0}
        q.precision = m.MHD_FP32
        pbs.append(q)
    cfgs = [m.Config.from_problem(q) for q in pbs]
    ens = m.Ensemble(cfgs)
    for b, q in enumerate(pbs):
        ens.set_state(b, torch.from_numpy(q.prim()).cuda(), kind=m.MHD_PRIM)
    ens.autotune(1)
    ens.step(10)
    for b, q in enumerate(pbs):
        s = m.MHD(cfgs[b])
        s.set_state(torch.from_numpy(q.prim()).cuda(), kind=m.MHD_PRIM)
        for _ in range(10):
            s.step()
        assert bool((ens.get_state(b) == s.get_state()).all()), f"box {b} (edge {sizes[b]})"
        assert ens.info(b)["t"] == s.step_info()["t"]
        del s


def test_adjoint_512_200_steps_against_central_differences():
    from test_gpu_adjoint import _J_frozen, _recorded, _rollout_grad
    pb = inputs.orszag_tang_2d(512, steps=200)
    dv = inputs.adjoint_perturbation(pb, seed=4)
    J, grad, _, _ = _rollout_grad(pb, dv, 200, 20)
    dts, chs = _recorded(pb, dv, 200)
    dirs = inputs.random_directions(dv.shape, 16, seed=4) * np.sqrt(dv.size) * 1e-3
    gnorm = float(np.sqrt(np.sum(grad * grad)))
    worst = 0.0
    for d in dirs:
        ad = float(np.sum(grad * d))
        scale = gnorm * float(np.sqrt(np.sum(d * d)))
        best = np.inf
        for eps in (1e-4, 1e-5, 1e-6):
            fd = (_J_frozen(pb, dv + eps * d, dts, chs)
                  - _J_frozen(pb, dv - eps * d, dts, chs)) / (2 * eps)
            best = min(best, abs(fd - ad) / scale)
        worst = max(worst, best)
    print("adjoint 512^2 x 200 steps: worst |fd - ad| / (|grad J| |d|) =", worst)
    assert worst < 1e-6, worst
