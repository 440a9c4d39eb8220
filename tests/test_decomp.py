"""Host logic of the decomposed grid (paper_2510_24175_gb300/decomp.py), on
the CPU: the block geometry and neighbours, the halo exchange through
torch.distributed with gloo ranks (which neighbour's data lands in which halo,
also when one rank is the neighbour on both sides), and the whole method run
by the oracle on 2 x 2 blocks (four gloo ranks): ghost zones filled through
that exchange -- faces, edges and corners, the 26 neighbours of a 3-D block
(Section 3.2), by exchanging the dimensions one after another over the
already padded extents -- must equal the oracle's own ghost fill of the
undecomposed grid, and the gathered result of the steps must equal the
undecomposed run bitwise."""
import os
import socket

import numpy as np
import pytest

from paper_2510_24175_gb300.decomp import OPPOSITE, Decomposition

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HALO, PER, OUT = 2, 0, 1


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_block_geometry_and_neighbours():
    dec = Decomposition((40, 24, 21), (2, 2, 3), (PER, PER, OUT, OUT, PER, PER))
    assert dec.nblocks == 12
    cover = np.zeros((21, 24, 40), dtype=int)
    for r in range(12):
        assert dec.rank_of(dec.coords(r)) == r
        lo, hi = dec.extent(r)
        cover[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] += 1
    assert (cover == 1).all()
    assert dec.shape(0) == (20, 12, 7)
    # x periodic with two blocks: both x neighbours of block 0 are block 1
    assert dec.neighbour(0, 0) == dec.neighbour(0, 1) == 1
    # y outflow: the low block has no low neighbour, the high block no high one
    assert dec.neighbour(0, 2) is None and dec.neighbour(0, 3) == 2
    assert dec.neighbour(2, 3) is None
    assert dec.local_bc(0) == (HALO, HALO, OUT, HALO, HALO, HALO)
    # z periodic with three blocks: wrap
    assert dec.neighbour(0, 4) == 8 and dec.neighbour(8, 5) == 0
    # neighbours are mutual across opposite faces
    for r in range(12):
        for f in range(6):
            nb = dec.neighbour(r, f)
            if nb is not None:
                assert dec.neighbour(nb, OPPOSITE[f]) == r
                s1, s2 = dec.shape(r), dec.shape(nb)
                assert all(s1[e] == s2[e] for e in range(3) if e != f >> 1)
    # one periodic block: no halo unless forced, then its own neighbour
    one = Decomposition((8, 8, 8), (1, 1, 1))
    assert one.halo_faces(0) == []
    forced = Decomposition((8, 8, 8), (1, 1, 1), force_halo=True)
    assert all(forced.neighbour(0, f) == 0 for f in range(6))
    U = np.arange(9 * 21 * 24 * 40, dtype=float).reshape(9, 21, 24, 40)
    back = dec.gather([dec.scatter(U, r) for r in range(12)], np.zeros_like(U))
    np.testing.assert_array_equal(back, U)


def test_config_validation_of_halo_faces():
    import paper_2510_24175_gb300 as m
    m.lib()
    import ctypes
    b = ctypes.c_size_t()
    for ok in (m.Config(n=(16, 16, 16), bc=(HALO, HALO, OUT, HALO, PER, PER)),
               m.Config(n=(16, 16, 16), bc=(HALO,) * 6, limiter=m.MHD_LIM_WENOZ, rk_order=3,
                        precision=m.MHD_FP32)):
        assert m.lib().mhd_workspace_bytes(ctypes.byref(ok.c()), ctypes.byref(b)) == m.MHD_OK
    for bad in (m.Config(n=(16, 16, 1), bc=(HALO, HALO, PER, PER, PER, PER)),   # 2-D
                m.Config(n=(16, 16, 16), bc=(HALO, PER, PER, PER, PER, PER)),   # periodic pair
                m.Config(n=(16, 16, 16), bc=(HALO,) * 6, divb=m.MHD_DIVB_CT),
                m.Config(n=(16, 16, 16), bc=(HALO,) * 6, flags=m.MHD_FLAG_ADJOINT)):
        assert m.lib().mhd_workspace_bytes(ctypes.byref(bad.c()), ctypes.byref(b)) == \
            m.MHD_ERR_INVALID


# ------------------------------------------------------------ gloo ranks --
def _init(rank, world, port):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _exchange_worker(rank, world, port, dims, bc):
    import torch
    dist = _init(rank, world, port)
    from paper_2510_24175_gb300.decomp import Decomposition, exchange
    dec = Decomposition((12, 10, 8), dims, bc)
    faces = dec.halo_faces(rank)
    send = {f: torch.full((5,), float(100 * rank + f)) for f in faces}
    recv = {f: torch.full((5,), -1.0) for f in faces}
    exchange(dec, rank, send, recv)
    for f in faces:
        nb = dec.neighbour(rank, f)
        assert torch.all(recv[f] == float(100 * nb + OPPOSITE[f])), (rank, f, recv[f])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("dims,bc", [((1, 2, 2), (PER,) * 6),
                                     ((2, 2, 1), (OUT, OUT, PER, PER, PER, PER)),
                                     ((4, 1, 1), (PER,) * 6)])
def test_exchange_delivers_each_neighbours_boundary(dims, bc):
    import torch.multiprocessing as mp
    world = dims[0] * dims[1] * dims[2]
    mp.start_processes(_exchange_worker, args=(world, _free_port(), dims, bc), nprocs=world,
                       join=True, start_method="spawn")


def _fill_padded(dec, rank, U, g, global_bc):
    """The block's padded array: interior U, ghosts dimension by dimension
    (x, then y over the x-padded extent, then z over both), each from the
    neighbour through the exchange or by the boundary rule."""
    import torch
    from paper_2510_24175_gb300.decomp import exchange
    nz, ny, nx = U.shape[1:]
    P = np.zeros((9, nz + 2 * g, ny + 2 * g, nx + 2 * g))
    P[:, g:-g, g:-g, g:-g] = U
    for d in range(3):
        axis = 3 - d
        # extent along the other axes: padded for earlier dimensions
        sl = [slice(None)] + [slice(g, -g)] * 3
        for e in range(d):
            sl[3 - e] = slice(None)
        n = P.shape[axis] - 2 * g
        send, recv = {}, {}
        for side in (0, 1):
            f = 2 * d + side
            if dec.neighbour(rank, f) is None:
                continue
            s = list(sl)
            s[axis] = slice(n, n + g) if side else slice(g, 2 * g)
            send[f] = torch.from_numpy(np.ascontiguousarray(P[tuple(s)]))
            recv[f] = torch.empty_like(send[f])
        exchange(dec, rank, send, recv, dims=(d,))
        for side in (0, 1):
            f = 2 * d + side
            s = list(sl)
            s[axis] = slice(n + g, n + 2 * g) if side else slice(0, g)
            if f in recv:
                P[tuple(s)] = recv[f].numpy()
            elif global_bc[f] == PER:  # an unsplit periodic dimension: wrap in the block
                src = list(sl)
                src[axis] = slice(g, 2 * g) if side else slice(n, n + g)
                P[tuple(s)] = P[tuple(src)]
            else:  # an outflow end: the nearest interior cell
                src = list(sl)
                src[axis] = slice(n + g - 1, n + g) if side else slice(g, g + 1)
                P[tuple(s)] = np.repeat(P[tuple(src)], g, axis=axis)
    return P


def _oracle_blocks_worker(rank, world, port, dims, bc, lim, rk, nsteps, out_path):
    import torch
    dist = _init(rank, world, port)
    import oracle as orc
    from paper_2510_24175_gb300.decomp import Decomposition
    from paper_2510_24175_gb300.inputs import Problem
    pb = Problem("random_smooth", (14, 12, 10), seed=53, bc=bc, limiter=lim, rk_order=rk)
    kw = dict(gamma=pb.gamma, glm_alpha=pb.glm_alpha, limiter=pb.limiter, cfl=pb.cfl,
              rk_order=pb.rk_order)
    G = orc.Grid(n=pb.n, dx=pb.dx, bc=pb.bc, **kw)
    dec = Decomposition(pb.n, dims, bc)
    U_full = orc.prim_to_cons(pb.prim(), pb.gamma)
    U = np.ascontiguousarray(dec.scatter(U_full, rank))
    L = orc.Grid(n=dec.shape(rank), dx=pb.dx, bc=tuple(1 if b == HALO else b
                                                        for b in dec.local_bc(rank)), **kw)
    g = G.ghost
    # the padded block equals the oracle's ghost fill of the undecomposed grid
    P = _fill_padded(dec, rank, U, g, bc)
    lo, hi = dec.extent(rank)
    ref = orc.fill_ghosts(U_full, G)[:, lo[2]:hi[2] + 2 * g, lo[1]:hi[1] + 2 * g,
                                     lo[0]:hi[0] + 2 * g]
    np.testing.assert_array_equal(P, ref)
    inv = sum(1.0 / pb.dx[d] for d in range(3))
    for _ in range(nsteps):
        lam = torch.tensor([orc.max_speed(U, L)], dtype=torch.float64)
        dist.all_reduce(lam, op=dist.ReduceOp.MAX)
        ch = float(lam[0])
        dt = pb.cfl / (ch * inv)
        W = orc.stage_padded(_fill_padded(dec, rank, U, g, bc), L, dt, ch, 1)
        if rk == 3:
            W = orc.stage_padded(_fill_padded(dec, rank, W, g, bc), L, dt, ch, 2, Un=U)
            U = orc.stage_padded(_fill_padded(dec, rank, W, g, bc), L, dt, ch, 3, Un=U,
                                 damp=True)
        else:
            U = orc.stage_padded(_fill_padded(dec, rank, W, g, bc), L, dt, ch, 2, Un=U,
                                 damp=True)
    parts = [torch.empty(0, dtype=torch.float64) for _ in range(world)]
    mine = torch.from_numpy(np.ascontiguousarray(U).ravel())
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([mine.numel()]))
    parts = [torch.empty(int(s), dtype=torch.float64) for s in sizes]
    dist.all_gather(parts, mine)
    if rank == 0:
        blocks = [p.numpy().reshape((9,) + tuple(reversed(dec.shape(r))))
                  for r, p in enumerate(parts)]
        np.save(out_path, dec.gather(blocks, np.zeros_like(U_full)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("lim,rk", [(2, 2), (3, 3)], ids=["plm_rk2", "wenoz_rk3"])
@pytest.mark.parametrize("bc", [(PER,) * 6, (PER, PER, OUT, OUT, PER, PER)],
                         ids=["periodic", "outflow_y"])
def test_oracle_on_2x2_blocks_is_bitwise_the_undecomposed_run(tmp_path, bc, lim, rk):
    import torch.multiprocessing as mp
    import oracle as orc
    from paper_2510_24175_gb300.inputs import Problem
    out = str(tmp_path / "blocks.npy")
    nsteps = 2
    mp.start_processes(_oracle_blocks_worker,
                       args=(4, _free_port(), (1, 2, 2), bc, lim, rk, nsteps, out), nprocs=4,
                       join=True, start_method="spawn")
    pb = Problem("random_smooth", (14, 12, 10), seed=53, bc=bc, limiter=lim, rk_order=rk)
    G = orc.Grid(n=pb.n, dx=pb.dx, gamma=pb.gamma, glm_alpha=pb.glm_alpha, limiter=lim,
                 bc=bc, cfl=pb.cfl, rk_order=rk)
    ref = orc.run(orc.prim_to_cons(pb.prim(), pb.gamma), G, nsteps)
    np.testing.assert_array_equal(np.load(out), ref.U)
