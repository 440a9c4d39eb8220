"""mhd_step_n (n CFL steps replayed from one captured CUDA graph) gives bit
for bit the states, time and step count of n mhd_step(ctx, 0, 0) calls: the
graph holds the same launches.  Covers graph reuse and re-capture, a 1-D
run past t_end (the clamped last step and the no-op steps after it), FP32,
WENO-Z + SSP-RK3, constrained transport, the per-launch fallback while
profiling, and the argument checks."""
import numpy as np
import pytest

from paper_2510_24175_gb300 import inputs

pytestmark = pytest.mark.gpu


def _mhd():
    import paper_2510_24175_gb300 as m
    return m


def _pair(pb, precision=None, ct=False):
    import torch
    m = _mhd()
    cfg = m.Config.from_problem(pb) if precision is None else \
        m.Config.from_problem(pb, precision=precision)
    out = []
    for _ in range(2):
        s = m.MHD(cfg)
        s.set_state(torch.from_numpy(pb.prim()).cuda(), kind=m.MHD_PRIM)
        if ct:
            s.set_face_field(torch.from_numpy(pb.faces()).cuda())
        out.append(s)
    return out


def _same(a, b):
    assert a.step_info() == b.step_info()
    np.testing.assert_array_equal(a.get_state().cpu().numpy(), b.get_state().cpu().numpy())


@pytest.mark.parametrize("case", ["fp64_3d", "fp32_3d", "wenoz_rk3", "ct"])
def test_graph_steps_equal_single_steps(case):
    m = _mhd()
    pb = inputs.orszag_tang_3d(8).with_n((40, 24, 16))
    prec = None
    if case == "fp32_3d":
        prec = m.MHD_FP32
    if case == "wenoz_rk3":
        pb.limiter, pb.rk_order = m.MHD_LIM_WENOZ, 3
    if case == "ct":
        pb.divb = m.MHD_DIVB_CT
    a, b = _pair(pb, prec, ct=case == "ct")
    for n in (3, 3, 5):  # capture, reuse, re-capture
        a.step_n(n)
        for _ in range(n):
            b.step()
        _same(a, b)


def test_graph_steps_past_t_end():
    pb = inputs.brio_wu(256)
    pb.t_end = 0.02
    a, b = _pair(pb)
    n = 0
    while b.step_info()["t"] < pb.t_end:
        b.step()
        n += 1
    for _ in range(4):  # no-op steps at t_end
        b.step()
    a.step_n(n + 4)
    _same(a, b)
    assert a.step_info()["t"] == pb.t_end


def test_graph_steps_with_profiling_and_argument_checks():
    m = _mhd()
    pb = inputs.orszag_tang_3d(8).with_n((32, 16, 8))
    a, b = _pair(pb)
    a.profile(True)
    a.step_n(4)
    counts = a.profile_read()
    a.profile(False)
    assert counts["stage1"][0] == 4 and counts["stage2"][0] == 4
    for _ in range(4):
        b.step()
    _same(a, b)
    a.step_n(0)
    _same(a, b)
    with pytest.raises(m.MHDError) as e:
        a.step_n(-1)
    assert e.value.code == m.MHD_ERR_INVALID


def test_stage1_after_graph_steps():
    """mhd_get_stage1 after mhd_step_n returns the last step's first stage,
    bitwise that of the same steps taken one by one, also when the captured
    graph is replayed after a new set_state."""
    import torch
    m = _mhd()
    pb = inputs.orszag_tang_3d(8).with_n((32, 16, 8))
    a, b = _pair(pb)
    V = torch.from_numpy(pb.prim()).cuda()
    for rep in range(2):  # capture, then replay after set_state
        if rep:
            a.set_state(V, kind=m.MHD_PRIM)
            b.set_state(V, kind=m.MHD_PRIM)
            with pytest.raises(m.MHDError) as e:
                a.get_stage1()
            assert e.value.code == m.MHD_ERR_STATE
        a.step_n(3)
        for _ in range(3):
            b.step()
        _same(a, b)
        np.testing.assert_array_equal(a.get_stage1().cpu().numpy(),
                                      b.get_stage1().cpu().numpy())
