"""Constrained transport on the GPU (the div-B control of the paper's
weak-scaling runs, Section 4.2) against the oracle's constrained transport:
state and face field element by element after several steps (FP64: 1e-12
relative L1 per variable / face component), for PLM and WENO-Z, RK2 and
SSP-RK3, on ragged grids that span several tiles; the face divergence stays
at round-off; FP32 at its stated tolerance; the face-field entry points and
the configurations constrained transport rejects."""
import numpy as np
import pytest

import oracle as orc
from paper_2510_24175_gb300 import inputs
from parity_util import gpu_run, grid_of, rel_l1

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


def _ct_gpu(pb, nsteps, precision=None):
    import torch
    import paper_2510_24175_gb300 as m
    s = m.MHD(m.Config.from_problem(pb, precision=precision))
    s.set_state(torch.from_numpy(pb.prim()).cuda(), kind=m.MHD_PRIM)
    s.set_face_field(torch.from_numpy(pb.faces()).cuda())
    for _ in range(nsteps):
        s.step()
    info = s.step_info()
    return s, s.get_state().cpu().numpy(), s.get_face_field().cpu().numpy(), info


def _ct_oracle(pb, nsteps):
    g = grid_of(pb)
    return orc.ct_run(orc.prim_to_cons(pb.prim(), pb.gamma), pb.faces(), g, nsteps)


def _face_rel(a, b, floor=1e-3):
    """Per component relative L1, the denominator floored at floor x the
    largest component's L1 (FP32: 0.1, as for the state)."""
    num = np.abs(a - b).reshape(3, -1).sum(axis=1)
    den = np.abs(b).reshape(3, -1).sum(axis=1)
    return num / np.maximum(den, floor * den.max())


@pytest.mark.parametrize("n,lim,rk", [
    ((40, 20, 13), orc.LIM_MC, 2),
    ((37, 18, 11), orc.LIM_MINMOD, 3),
    ((36, 14, 12), orc.LIM_WENOZ, 3),
    ((35, 9, 10), orc.LIM_WENOZ, 2),
])
def test_ct_matches_oracle(n, lim, rk):
    pb = inputs.ct_random(n, seed=13)
    pb.limiter, pb.rk_order = lim, rk
    steps = 6
    ref = _ct_oracle(pb, steps)
    _, U, b, info = _ct_gpu(pb, steps)
    assert info["steps"] == steps and abs(info["t"] - ref.t) <= 1e-14 * ref.t
    assert np.all(rel_l1(U, ref.U) <= TOL64), rel_l1(U, ref.U)
    assert np.all(_face_rel(b, ref.b) <= TOL64), _face_rel(b, ref.b)
    assert np.abs(U[8]).max() == 0.0


@pytest.mark.parametrize("lim,rk", [(orc.LIM_MC, 2), (orc.LIM_WENOZ, 3)])
def test_ct_orszag_tang_matches_oracle(lim, rk):
    pb = inputs.orszag_tang_3d_ct(24, limiter=lim, rk_order=rk).with_n((40, 24, 20))
    ref = _ct_oracle(pb, 5)
    _, U, b, _ = _ct_gpu(pb, 5)
    assert np.all(rel_l1(U, ref.U) <= TOL64), rel_l1(U, ref.U)
    assert np.all(_face_rel(b, ref.b) <= TOL64), _face_rel(b, ref.b)


def test_ct_plane_parallel_shock_pairs():
    """Two Brio-Wu tubes on a 3-D grid along each axis: the GPU's CT run
    against the oracle's CT run (which the oracle pins reduce exactly to the
    1-D scheme)."""
    for axis in range(3):
        pb = inputs.shock_pair(64, 6, axis=axis)
        ref = _ct_oracle(pb, 20)
        _, U, b, _ = _ct_gpu(pb, 20)
        assert np.all(rel_l1(U, ref.U) <= TOL64), (axis, rel_l1(U, ref.U))
        assert np.all(_face_rel(b, ref.b) <= TOL64), (axis, _face_rel(b, ref.b))


def test_ct_divergence_stays_at_round_off_on_gpu():
    pb = inputs.ct_random((48, 40, 36), seed=17)
    s, U, b, _ = _ct_gpu(pb, 0)
    scale = np.abs(b).max() / min(pb.dx)
    d0 = s.divb_max()
    # the input field's own divergence: round-off of the face averages
    assert d0 <= 1e-13 * scale
    ref = np.abs(orc.ct_divb(b, grid_of(pb))).max()
    assert abs(d0 - ref) <= 1e-15 * scale
    for _ in range(30):
        s.step()
    assert s.divb_max() <= d0 + 1e-13 * scale
    b1 = s.get_face_field().cpu().numpy()
    assert np.abs(b1 - b).max() > 1e-3 * np.abs(b).max()
    # the face-field sums (periodic) are conserved
    assert np.abs(b1.sum(axis=(1, 2, 3)) - b.sum(axis=(1, 2, 3))).max() <= 1e-10


def test_ct_fp32_against_fp64_oracle():
    pb = inputs.orszag_tang_3d_ct(24).with_n((40, 24, 16))
    ref = _ct_oracle(pb, 4)
    s, U, b, _ = _ct_gpu(pb, 4, precision=1)
    assert np.all(rel_l1(U, ref.U, floor=0.1) <= TOL32), rel_l1(U, ref.U, floor=0.1)
    assert np.all(_face_rel(b, ref.b, floor=0.1) <= TOL32), _face_rel(b, ref.b, floor=0.1)
    scale = np.abs(b).max() / min(pb.dx)
    assert s.divb_max() <= 1e-5 * scale


def test_set_face_field_keeps_pressure():
    import torch
    import paper_2510_24175_gb300 as m
    pb = inputs.ct_random((16, 12, 10), seed=19)
    V = pb.prim()
    b = pb.faces()
    s = m.MHD(m.Config.from_problem(pb))
    # a state whose B differs from the face means: B replaced, p kept
    V2 = V.copy()
    V2[4:7] += 0.1
    s.set_state(torch.from_numpy(V2).cuda(), kind=m.MHD_PRIM)
    s.set_face_field(b)
    W = s.get_state(kind=m.MHD_PRIM).cpu().numpy()
    assert np.abs(W[4:7] - V[4:7]).max() <= 1e-15
    assert np.abs(W[7] - V2[7]).max() <= 1e-12 * np.abs(V2[7]).max()
    # a state whose B equals the face means is unchanged bit for bit
    s.set_state(torch.from_numpy(V).cuda(), kind=m.MHD_PRIM)
    U0 = s.get_state().cpu().numpy()
    s.set_face_field(torch.from_numpy(b).cuda())
    assert np.array_equal(s.get_state().cpu().numpy(), U0)
    assert np.array_equal(s.get_face_field().cpu().numpy(), b)
    host = np.empty_like(b)
    s.get_face_field(host)
    assert np.array_equal(host, b)


def test_ct_rejections_and_state_rules():
    import torch
    import paper_2510_24175_gb300 as m
    for kw in ({"n": (16, 16, 1)}, {"n": (16, 16, 16), "bc": (1,) * 6},
               {"n": (16, 16, 16), "flags": m.MHD_FLAG_ADJOINT}):
        with pytest.raises(m.MHDError):
            m.MHD(m.Config(divb=m.MHD_DIVB_CT, **kw))
    with pytest.raises(m.MHDError):
        m.Ensemble([m.Config(n=(16, 16, 16), precision=m.MHD_FP32, divb=m.MHD_DIVB_CT)])
    pb = inputs.ct_random((16, 12, 10))
    s = m.MHD(m.Config.from_problem(pb))
    with pytest.raises(m.MHDError):
        s.set_face_field(pb.faces())  # before set_state
    s.set_state(torch.from_numpy(pb.prim()).cuda(), kind=m.MHD_PRIM)
    with pytest.raises(m.MHDError) as e:
        s.step()  # no face field yet
    assert e.value.code == m.MHD_ERR_STATE
    s.set_face_field(pb.faces())
    s.step()
    s.step_info()
    g = m.MHD(m.Config(n=pb.n))
    with pytest.raises(m.MHDError):
        g.set_face_field(pb.faces())
    with pytest.raises(m.MHDError):
        g.divb_max()
