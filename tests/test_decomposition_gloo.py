"""Domain decomposition of the Runge-Kutta step across ranks (the multi-GPU layout:
one subdomain per rank, a ghost-zone exchange before every stage -- the
paper's boundary exchange, Section 3.2 -- and a max-allreduce of the wave
speed for the common dt and c_h), exercised with world_size 2 gloo ranks on
the CPU with the oracle doing each rank's stage.  The gathered result must be
bitwise equal to the undecomposed run: the per-cell arithmetic is identical
once the ghost values are, and a max is exact.  Both schemes: PLM + RK2
(two ghost planes per stage) and the paper's WENO-Z + SSP-RK3 (three ghost
planes, three exchanges per step)."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _pad_xy(U, bc_x, bc_y, gw):
    """Ghost fill of x and y (undivided dimensions) by the boundary rule."""
    mode = {0: "wrap", 1: "edge"}
    U = np.pad(U, [(0, 0), (0, 0), (0, 0), (gw, gw)], mode=mode[bc_x])
    return np.pad(U, [(0, 0), (0, 0), (gw, gw), (0, 0)], mode=mode[bc_y])


SCHEMES = {"plm_rk2": (2, 2), "wenoz_rk3": (3, 3)}  # limiter, rk_order


def _problem(bc_z, scheme):
    from paper_2510_24175_gb300.inputs import Problem
    lim, rk = SCHEMES[scheme]
    return Problem("random_smooth", (10, 8, 12), seed=17, bc=(0, 0, 1, 1, bc_z, bc_z),
                   limiter=lim, rk_order=rk)


def _worker(rank, world, port, bc_z, scheme, nsteps, out_path):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as orc

    pb = _problem(bc_z, scheme)
    U_full = orc.prim_to_cons(pb.prim(), pb.gamma)
    nzl = pb.n[2] // world
    U = U_full[:, rank * nzl:(rank + 1) * nzl].copy()
    g = orc.Grid(n=(pb.n[0], pb.n[1], nzl), dx=pb.dx, gamma=pb.gamma, glm_alpha=pb.glm_alpha,
                 limiter=pb.limiter, bc=pb.bc, cfl=pb.cfl, rk_order=pb.rk_order)
    gw = g.ghost
    inv = 1.0 / pb.dx[0] + 1.0 / pb.dx[1] + 1.0 / pb.dx[2]

    def exchange(W):
        """Padded array: x/y ghosts by the boundary rule, z ghosts (gw planes
        a side) from the neighbouring ranks (or the boundary rule at the
        global ends)."""
        P = _pad_xy(W, pb.bc[0], pb.bc[2], gw)
        mine = torch.from_numpy(np.ascontiguousarray(np.concatenate([P[:, :gw], P[:, -gw:]], 1)))
        allb = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(allb, mine)
        below, above = (rank - 1) % world, (rank + 1) % world
        lo = allb[below].numpy()[:, gw:]   # top gw planes of the rank below
        hi = allb[above].numpy()[:, :gw]   # bottom gw planes of the rank above
        if bc_z == 1 and rank == 0:
            lo = np.repeat(P[:, :1], gw, axis=1)
        if bc_z == 1 and rank == world - 1:
            hi = np.repeat(P[:, -1:], gw, axis=1)
        return np.concatenate([lo, P, hi], axis=1)

    for _ in range(nsteps):
        lam = torch.tensor([orc.max_speed(U, g)], dtype=torch.float64)
        dist.all_reduce(lam, op=dist.ReduceOp.MAX)
        ch = float(lam[0])
        dt = pb.cfl / (ch * inv)
        U1 = orc.stage_padded(exchange(U), g, dt, ch, 1)
        if pb.rk_order == 3:
            U2 = orc.stage_padded(exchange(U1), g, dt, ch, 2, Un=U)
            U = orc.stage_padded(exchange(U2), g, dt, ch, 3, Un=U, damp=True)
        else:
            U = orc.stage_padded(exchange(U1), g, dt, ch, 2, Un=U, damp=True)

    parts = [torch.empty(U.shape, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, torch.from_numpy(U))
    if rank == 0:
        np.save(out_path, np.concatenate([p.numpy() for p in parts], axis=1))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("scheme", sorted(SCHEMES))
@pytest.mark.parametrize("bc_z", [0, 1], ids=["periodic_z", "outflow_z"])
def test_two_rank_decomposition_is_bitwise_equal(tmp_path, bc_z, scheme):
    import torch.multiprocessing as mp
    import oracle as orc
    out = str(tmp_path / "decomposed.npy")
    nsteps = 3
    mp.start_processes(_worker, args=(2, _free_port(), bc_z, scheme, nsteps, out), nprocs=2,
                       join=True, start_method="spawn")
    got = np.load(out)
    pb = _problem(bc_z, scheme)
    g = orc.Grid(n=pb.n, dx=pb.dx, gamma=pb.gamma, glm_alpha=pb.glm_alpha, limiter=pb.limiter,
                 bc=pb.bc, cfl=pb.cfl, rk_order=pb.rk_order)
    ref = orc.run(orc.prim_to_cons(pb.prim(), pb.gamma), g, nsteps)
    np.testing.assert_array_equal(got, ref.U)
