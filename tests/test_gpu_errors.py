"""Error paths of the C ABI, with every fault injected on the host: a
non-finite state, calls out of order, bad arguments and an undersized
workspace.  Device-side numerics faults come back as MHD_ERR_NONFINITE from
the next synchronising call; the step that meets a non-finite time step is a
no-op, so the state stays inspectable.  No kernel traps or spins."""
import ctypes

import numpy as np
import pytest

from paper_2510_24175_gb300.inputs import Problem

pytestmark = pytest.mark.gpu


def _mhd():
    import paper_2510_24175_gb300 as m
    return m


def test_nonfinite_state_is_reported_and_step_becomes_noop():
    import torch
    m = _mhd()
    pb = Problem("random_smooth", (16, 8, 4), seed=2)
    s = m.MHD(m.Config.from_problem(pb))
    V = pb.prim()
    V[7, 1, 2, 3] = np.nan  # pressure of one cell
    s.set_state(torch.from_numpy(V).cuda(), kind=m.MHD_PRIM)
    with pytest.raises(m.MHDError) as e:
        s.dt()
    assert e.value.code == m.MHD_ERR_NONFINITE
    before = s.get_state().cpu().numpy()
    s.step()  # dt from a NaN wave speed: flagged, dt = 0
    with pytest.raises(m.MHDError) as e:
        s.step_info()
    assert e.value.code == m.MHD_ERR_NONFINITE
    after = s.get_state().cpu().numpy()
    np.testing.assert_array_equal(np.isnan(after), np.isnan(before))
    np.testing.assert_array_equal(after[~np.isnan(after)], before[~np.isnan(before)])
    assert s.counters()["status"] != 0


def test_nan_appearing_during_a_step_is_reported():
    import torch
    m = _mhd()
    pb = Problem("random_smooth", (16, 8, 4), seed=3)
    s = m.MHD(m.Config.from_problem(pb))
    V = pb.prim()
    V[8, 0, 0, 0] = np.inf  # psi: the wave speed stays finite, the update does not
    s.set_state(torch.from_numpy(V).cuda(), kind=m.MHD_PRIM)
    s.step(1e-3, 1.0)
    with pytest.raises(m.MHDError) as e:
        s.step_info()
    assert e.value.code == m.MHD_ERR_NONFINITE


def test_calls_out_of_order_and_bad_arguments():
    import torch
    m = _mhd()
    pb = Problem("random_smooth", (8, 8, 1), seed=4)
    s = m.MHD(m.Config.from_problem(pb))
    with pytest.raises(m.MHDError) as e:
        s.step()
    assert e.value.code == m.MHD_ERR_STATE
    with pytest.raises(m.MHDError) as e:
        s.dt()
    assert e.value.code == m.MHD_ERR_STATE
    s.set_state(torch.from_numpy(pb.prim()).cuda(), kind=m.MHD_PRIM)
    for dt, ch in [(float("nan"), 1.0), (1e-3, float("inf"))]:
        with pytest.raises(m.MHDError) as e:
            s.step(dt, ch)
        assert e.value.code == m.MHD_ERR_INVALID
    U = s.get_state()
    lam = torch.zeros_like(U)
    with pytest.raises(m.MHDError) as e:  # context created without the adjoint flag
        s.adjoint_step(U, lam, torch.empty_like(U), 1e-3, 1.0)
    assert e.value.code == m.MHD_ERR_STATE
    with pytest.raises(m.MHDError) as e:
        s.get_state(np.empty(s.shape), kind=m.MHD_PRIM)  # primitive output needs device memory
    assert e.value.code == m.MHD_ERR_INVALID


def test_undersized_or_misaligned_workspace_is_rejected():
    import torch
    m = _mhd()
    cfg = m.Config(n=(32, 16, 8)).c()
    need = m.mhd_workspace_bytes(cfg)
    small = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    ctx = ctypes.c_void_p()
    rc = m.lib().mhd_create(ctypes.byref(cfg), ctypes.c_void_p(small.data_ptr()), need - 256,
                            None, ctypes.byref(ctx))
    assert rc == m.MHD_ERR_NOMEM
    big = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    rc = m.lib().mhd_create(ctypes.byref(cfg), ctypes.c_void_p(big.data_ptr() + 8), need, None,
                            ctypes.byref(ctx))
    assert rc == m.MHD_ERR_NOMEM


def test_step_reaches_t_end_exactly_then_stops():
    import torch
    m = _mhd()
    pb = Problem("random_smooth", (16, 8, 1), seed=5, t_end=0.01)
    s = m.MHD(m.Config.from_problem(pb))
    s.set_state(torch.from_numpy(pb.prim()).cuda(), kind=m.MHD_PRIM)
    info = s.run(1000, t_end=pb.t_end)
    assert info["t"] == pytest.approx(0.01, abs=1e-15)
    U = s.get_state().cpu().numpy()
    s.step()  # at t_end: a zero-length step
    info2 = s.step_info()
    assert info2["t"] == info["t"] and info2["dt"] == 0.0
    np.testing.assert_array_equal(s.get_state().cpu().numpy(), U)
