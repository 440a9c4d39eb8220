"""Halo faces on the GPU: a grid decomposed into blocks, one context per
block, each stage reading its neighbours' boundary layers from halo buffers
(the paper's boundary exchange between processes, Section 3.2) and the
common dt / c_h from the maximum of the blocks' wave speeds.  Every block
must evolve bitwise as its cells do in one undecomposed context: the
per-cell arithmetic is the same and a maximum is exact.

Covered: splits along y and z (four blocks), along x and z, uneven blocks on
all three axes, outflow ends next to halo faces, PLM + RK2 and WENO-Z +
SSP-RK3, FP64 and FP32; a single block exchanging with itself (every face a
halo face); one rank of the distributed driver over NCCL (the exchange's
self-copy path and the allreduce of the wave speed); and the calls that
must be refused."""
import ctypes
import os
import socket

import numpy as np
import pytest

from paper_2510_24175_gb300.inputs import Problem

pytestmark = pytest.mark.gpu

NSTEPS = 3


def _reference(cfg, V, nsteps):
    import torch
    import paper_2510_24175_gb300 as m
    s = m.MHD(cfg)
    s.set_state(V, kind=m.MHD_PRIM)
    infos = []
    for _ in range(nsteps):
        s.step()
        infos.append(s.step_info())
    return s.get_state(), infos


CASES = {
    # name: (n, dims, bc, limiter, rk, precision)
    "yz_plm_fp64": ((40, 24, 20), (1, 2, 2), (0,) * 6, 2, 2, 0),
    "yz_plm_fp32": ((40, 24, 20), (1, 2, 2), (0,) * 6, 2, 2, 1),
    "xz_outflow_wenoz_rk3_fp64": ((70, 12, 20), (2, 1, 2), (0, 0, 1, 1, 1, 1), 3, 3, 0),
    "xz_outflow_wenoz_rk3_fp32": ((70, 12, 20), (2, 1, 2), (0, 0, 1, 1, 1, 1), 3, 3, 1),
    "uneven_xyz_minmod_fp64": ((37, 23, 19), (2, 2, 2), (0,) * 6, 1, 2, 0),
    "uneven_xyz_outflow_y": ((37, 23, 19), (2, 3, 2), (0, 0, 1, 1, 0, 0), 2, 2, 0),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_blocks_evolve_bitwise_as_the_undecomposed_grid(name):
    import torch
    import paper_2510_24175_gb300 as m
    from paper_2510_24175_gb300.decomp import LocalBlocks
    n, dims, bc, lim, rk, prec = CASES[name]
    pb = Problem("random_smooth", n, seed=29, bc=bc, limiter=lim, rk_order=rk)
    cfg = m.Config.from_problem(pb, precision=prec)
    V = torch.from_numpy(pb.prim()).cuda()
    ref, infos = _reference(cfg, V, NSTEPS)
    lb = LocalBlocks(cfg, dims)
    lb.set_state(V, kind=m.MHD_PRIM)
    for _ in range(NSTEPS):
        lb.step()
    got = lb.get_state()
    assert torch.equal(got, ref), float((got - ref).abs().max())
    for b in lb.blocks:
        info = b.step_info()
        assert (info["t"], info["dt"], info["ch"]) == (infos[-1]["t"], infos[-1]["dt"],
                                                       infos[-1]["ch"])
        assert b.counters()["status"] == 0


@pytest.mark.parametrize("lim,rk", [(2, 2), (3, 3)])
def test_one_block_exchanging_with_itself_is_the_periodic_grid(lim, rk):
    """Every face a halo face whose neighbour is the block itself: the
    halo kernels reading the block's own boundary layers reproduce the
    periodic wrap of the plain kernels, bitwise."""
    import torch
    import paper_2510_24175_gb300 as m
    from paper_2510_24175_gb300.decomp import LocalBlocks
    pb = Problem("random_smooth", (40, 20, 12), seed=31, limiter=lim, rk_order=rk)
    cfg = m.Config.from_problem(pb)
    V = torch.from_numpy(pb.prim()).cuda()
    ref, _ = _reference(cfg, V, NSTEPS)
    lb = LocalBlocks(cfg, (1, 1, 1), force_halo=True)
    assert lb.dec.halo_faces(0) == list(range(6))
    lb.set_state(V, kind=m.MHD_PRIM)
    for _ in range(NSTEPS):
        lb.step()
    assert torch.equal(lb.get_state(), ref)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_distributed_block_on_one_rank_over_nccl():
    """The multi-GPU driver on a one-rank NCCL group: allreduce(MAX) of the
    wave-speed bits, packs into send buffers, the exchange (here the
    self-copy path) into the halo buffers, the halo stage kernels."""
    import torch
    import torch.distributed as dist
    import paper_2510_24175_gb300 as m
    from paper_2510_24175_gb300.decomp import DistributedBlock
    pb = Problem("random_smooth", (40, 20, 12), seed=37)
    cfg = m.Config.from_problem(pb)
    V = torch.from_numpy(pb.prim()).cuda()
    ref, _ = _reference(cfg, V, NSTEPS)
    store = dist.TCPStore("127.0.0.1", _free_port(), 1, True)
    dist.init_process_group("nccl", store=store, rank=0, world_size=1)
    try:
        blk = DistributedBlock(cfg, (1, 1, 1), 0, force_halo=True)
        blk.solver.set_state(V, kind=m.MHD_PRIM)
        for _ in range(NSTEPS):
            blk.step()
        assert torch.equal(blk.solver.get_state(), ref)
    finally:
        dist.destroy_process_group()


def test_halo_contexts_refuse_the_unstaged_calls_and_missing_buffers():
    import torch
    import paper_2510_24175_gb300 as m
    from paper_2510_24175_gb300.decomp import Decomposition
    pb = Problem("random_smooth", (40, 24, 20), seed=41)
    cfg = m.Config.from_problem(pb)
    dec = Decomposition(cfg.n, (1, 2, 1))
    s = m.MHD(dec.local_config(cfg, 0))
    s.set_state(torch.from_numpy(np.ascontiguousarray(dec.scatter(pb.prim(), 0))).cuda(),
                kind=m.MHD_PRIM)
    for call in (lambda: s.step(), lambda: s.step_n(2)):
        with pytest.raises(m.MHDError) as e:
            call()
        assert e.value.code == m.MHD_ERR_STATE
    s.step_begin()
    with pytest.raises(m.MHDError) as e:
        s.step_stage([None] * 6)
    assert e.value.code == m.MHD_ERR_INVALID
    with pytest.raises(m.MHDError) as e:  # a step is open
        s.lambda_max_into(torch.zeros(1, dtype=torch.int64, device="cuda"))
    assert e.value.code == m.MHD_ERR_STATE
    assert s.halo_bytes(2) == 9 * 2 * 20 * 40 * 8  # [9][nz][g][nx] FP64


def test_halo_pack_layout_matches_the_documented_slabs():
    """mhd_halo_pack of each face equals the g boundary layers of the state,
    laid out as the grid's SoA slab (checked with numpy slicing)."""
    import torch
    import paper_2510_24175_gb300 as m
    pb = Problem("random_smooth", (21, 13, 11), seed=43, limiter=3)  # g = 3
    cfg = m.Config.from_problem(pb)
    s = m.MHD(cfg)
    U = pb.prim()  # any array will do: set it as the conservative state
    s.set_state(torch.from_numpy(U).cuda())
    g = 3
    for f in range(6):
        buf = s.halo_buffer(f)
        s.halo_pack(f, buf)
        d, side = f >> 1, f & 1
        axis = 3 - d
        sl = [slice(None)] * 4
        nn = U.shape[axis]
        sl[axis] = slice(nn - g, nn) if side else slice(0, g)
        want = np.ascontiguousarray(U[tuple(sl)]).ravel()
        np.testing.assert_array_equal(buf.cpu().numpy(), want)
