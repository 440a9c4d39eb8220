"""mhd_step_host (one step of a host-resident state, copies overlapped with
the device work) gives bit for bit the state, time and step count of
mhd_set_state(host) + mhd_step + mhd_get_state(host): the same kernels do
the same per-cell arithmetic whatever the launch decomposition, and the
wave-speed maximum is order independent.  Covers the overlapped FP64 3-D
path (ragged z halves and slabs, output aliasing the input, CFL and given
dt / c_h), the sequential fallback (FP32, 2-D, nz < 8) and the rejection of
constrained transport."""
import numpy as np
import pytest

from paper_2510_24175_gb300 import inputs

pytestmark = pytest.mark.gpu


def _mhd():
    import paper_2510_24175_gb300 as m
    return m


def _pinned(shape):
    import torch
    return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()


def _reference(m, cfg, U0, nsteps, dt=0.0, ch=0.0):
    s = m.MHD(cfg)
    U = U0.copy()
    infos = []
    for _ in range(nsteps):
        s.set_state(U)
        s.step(dt, ch)
        out = np.empty_like(U)
        s.get_state(out)
        infos.append(s.step_info())
        U = out
    return U, infos


def _cons(m, pb, precision=None):
    """Conservative host state of a problem, via the library's own prim->cons."""
    import torch
    cfg = m.Config.from_problem(pb) if precision is None else \
        m.Config.from_problem(pb, precision=precision)
    s = m.MHD(cfg)
    s.set_state(torch.from_numpy(pb.prim()).cuda(), kind=m.MHD_PRIM)
    U = np.empty((9,) + tuple(pb.prim().shape[1:]))
    s.get_state(U)
    return cfg, U


@pytest.mark.parametrize("n", [(48, 40, 24), (40, 24, 13)])
def test_overlapped_fp64_equals_separate_calls(n):
    m = _mhd()
    pb = inputs.orszag_tang_3d(8).with_n(n)
    cfg, U0 = _cons(m, pb)
    ref, infos = _reference(m, cfg, U0, 3)
    s = m.MHD(cfg)
    U_in = _pinned(U0.shape)
    U_out = _pinned(U0.shape)
    U_in[...] = U0
    for k in range(3):
        s.step_host(U_in, U_out)
        info = s.step_info()
        assert info == infos[k], (info, infos[k])
        U_in[...] = U_out
    np.testing.assert_array_equal(U_out, ref)


def test_overlapped_output_may_alias_input_and_given_dt():
    m = _mhd()
    pb = inputs.orszag_tang_3d(8).with_n((32, 16, 16))
    cfg, U0 = _cons(m, pb)
    dt, ch = 1.3e-3, 2.5
    ref, _ = _reference(m, cfg, U0, 2, dt, ch)
    s = m.MHD(cfg)
    U = _pinned(U0.shape)
    U[...] = U0
    s.step_host(U, U, dt, ch)
    s.step_host(U, U, dt, ch)
    np.testing.assert_array_equal(U, ref)
    info = s.step_info()
    assert info["dt"] == dt and info["ch"] == ch


def test_pageable_buffers_give_the_same_result():
    m = _mhd()
    pb = inputs.orszag_tang_3d(8).with_n((32, 16, 16))
    cfg, U0 = _cons(m, pb)
    ref, _ = _reference(m, cfg, U0, 1)
    s = m.MHD(cfg)
    out = np.empty_like(U0)
    s.step_host(U0.copy(), out)
    np.testing.assert_array_equal(out, ref)


@pytest.mark.parametrize("case", ["fp32", "2d", "thin_z"])
def test_sequential_fallback_equals_separate_calls(case):
    m = _mhd()
    if case == "fp32":
        pb = inputs.orszag_tang_3d(8).with_n((32, 16, 16))
        cfg, U0 = _cons(m, pb, precision=m.MHD_FP32)
    elif case == "2d":
        pb = inputs.orszag_tang_2d(32)
        cfg, U0 = _cons(m, pb)
    else:
        pb = inputs.orszag_tang_3d(8).with_n((32, 16, 6))
        cfg, U0 = _cons(m, pb)
    ref, infos = _reference(m, cfg, U0, 2)
    s = m.MHD(cfg)
    U_in = _pinned(U0.shape)
    U_out = _pinned(U0.shape)
    U_in[...] = U0
    for k in range(2):
        s.step_host(U_in, U_out)
        assert s.step_info() == infos[k]
        U_in[...] = U_out
    np.testing.assert_array_equal(U_out, ref)


def test_constrained_transport_is_rejected():
    m = _mhd()
    pb = inputs.orszag_tang_3d(16)
    pb.divb = m.MHD_DIVB_CT
    cfg = m.Config.from_problem(pb)
    s = m.MHD(cfg)
    U = np.zeros((9,) + tuple(pb.prim().shape[1:]))
    with pytest.raises(m.MHDError) as e:
        s.step_host(U, U)
    assert e.value.code == m.MHD_ERR_INVALID
