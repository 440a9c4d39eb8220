"""A grid decomposed into blocks, one context per block (halo faces).

Section 3.2 of the paper: each process owns a block of the grid; before
every stage the ghost zones of the block's sides are exchanged with the
neighbouring processes (non-blocking MPI with up to 26 neighbours in 3-D),
and the time step needs the global maximum wave speed.  Here:

* ``Decomposition`` -- the blocks of a (px, py, pz) block grid, their
  extents, the neighbour across each face (periodic wrap or none at an
  outflow end) and each block's boundary conditions (``MHD_BC_HALO`` where a
  neighbour supplies the ghosts).
* ``exchange`` -- the halo exchange of one rank through ``torch.distributed``
  point-to-point operations, in a fixed phase order (per dimension: upward
  sends into the neighbours' low halos, then downward sends into their high
  halos), so the pairing is unambiguous with any backend; a face whose
  neighbour is the rank itself is a local copy.  Host logic only: it moves
  whatever tensors it is given (CUDA tensors over NCCL for the solver, CPU
  tensors over gloo in the tests).
* ``LocalBlocks`` -- every block in one process on one GPU: a halo buffer
  is filled by packing the neighbouring block's boundary straight into it.
* ``DistributedBlock`` -- one block per rank: halo buffers packed, exchanged
  with ``exchange`` and read by the next stage; the wave speed reduced with
  an allreduce(MAX) of its FP64 bit pattern.

The CUDA stage kernels read only face ghosts (each face flux uses cells along
its own axis), so six faces are exchanged; the oracle's padded stage in the
tests fills edges and corners too, by exchanging the dimensions one after
another over the already padded extents.  Every block evolves bitwise as its
cells do in the undecomposed grid (same per-cell arithmetic, exact maximum).
"""
from __future__ import annotations

from dataclasses import dataclass, replace

from . import MHD, MHD_BC_HALO, MHD_BC_PERIODIC, Config

OPPOSITE = [1, 0, 3, 2, 5, 4]


def _split(n: int, p: int):
    """[lo, hi) of each of p contiguous parts of n cells, as even as possible."""
    base, extra = divmod(n, p)
    out, lo = [], 0
    for r in range(p):
        h = base + (1 if r < extra else 0)
        out.append((lo, lo + h))
        lo += h
    return out


@dataclass
class Decomposition:
    """Blocks of a global grid of n = (nx, ny, nz) cells on a (px, py, pz)
    block grid; rank = ix + px (iy + py iz).  bc: the global boundary
    conditions (x-, x+, y-, y+, z-, z+).  force_halo: dimensions with a
    single periodic block still exchange halos (with the block itself), which
    exercises the halo path on one rank."""
    n: tuple
    dims: tuple
    bc: tuple = (MHD_BC_PERIODIC,) * 6
    force_halo: bool = False

    def __post_init__(self):
        self.n = tuple(int(v) for v in self.n)
        self.dims = tuple(int(v) for v in self.dims)
        assert len(self.n) == 3 and len(self.dims) == 3 and all(p >= 1 for p in self.dims)
        assert all(self.n[d] >= self.dims[d] for d in range(3))
        self.parts = [_split(self.n[d], self.dims[d]) for d in range(3)]

    @property
    def nblocks(self) -> int:
        return self.dims[0] * self.dims[1] * self.dims[2]

    def coords(self, rank: int):
        px, py, _ = self.dims
        return (rank % px, (rank // px) % py, rank // (px * py))

    def rank_of(self, c) -> int:
        px, py, _ = self.dims
        return c[0] + px * (c[1] + py * c[2])

    def extent(self, rank: int):
        """(lo, hi) index triples of the block's cells."""
        c = self.coords(rank)
        lo = tuple(self.parts[d][c[d]][0] for d in range(3))
        hi = tuple(self.parts[d][c[d]][1] for d in range(3))
        return lo, hi

    def shape(self, rank: int):
        lo, hi = self.extent(rank)
        return tuple(hi[d] - lo[d] for d in range(3))

    def _periodic(self, d: int) -> bool:
        return self.bc[2 * d] == MHD_BC_PERIODIC

    def exchanges(self, d: int) -> bool:
        """Whether the blocks exchange ghosts along dimension d."""
        return self.dims[d] > 1 or (self.force_halo and self._periodic(d) and self.n[d] > 1)

    def neighbour(self, rank: int, face: int):
        """The rank across face f (2 d + side), or None at an outflow end or
        along a dimension without exchange."""
        d, side = face >> 1, face & 1
        if not self.exchanges(d):
            return None
        c = list(self.coords(rank))
        c[d] += 1 if side else -1
        if c[d] < 0 or c[d] >= self.dims[d]:
            if not self._periodic(d):
                return None
            c[d] %= self.dims[d]
        return self.rank_of(c)

    def local_bc(self, rank: int):
        """The block's boundary conditions: MHD_BC_HALO across a neighbour,
        else the global rule."""
        return tuple(MHD_BC_HALO if self.neighbour(rank, f) is not None else self.bc[f]
                     for f in range(6))

    def halo_faces(self, rank: int):
        return [f for f in range(6) if self.neighbour(rank, f) is not None]

    def local_config(self, cfg: Config, rank: int) -> Config:
        """The block's configuration: its cells, its part of the domain, its
        boundary conditions, and the whole grid's cell size passed as given
        (the block's time step and flux divergence then round as the whole
        grid's do)."""
        lo, hi = self.extent(rank)
        dx = tuple((cfg.xmax[d] - cfg.xmin[d]) / cfg.n[d] if not (cfg.dx[d] > 0) else cfg.dx[d]
                   for d in range(3))
        return replace(cfg, n=self.shape(rank),
                       xmin=tuple(cfg.xmin[d] + lo[d] * dx[d] for d in range(3)),
                       xmax=tuple(cfg.xmin[d] + hi[d] * dx[d] for d in range(3)),
                       bc=self.local_bc(rank), dx=dx)

    def scatter(self, U, rank: int):
        """The block's part of a global array (..., nz, ny, nx)."""
        lo, hi = self.extent(rank)
        return U[..., lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]

    def gather(self, blocks, out):
        """Writes every block's array into out (..., nz, ny, nx)."""
        for r, B in enumerate(blocks):
            lo, hi = self.extent(r)
            out[..., lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = B
        return out


def exchange(dec: Decomposition, rank: int, send: dict, recv: dict, group=None,
             dims=(0, 1, 2)):
    """One rank's halo exchange.  send[f]: this rank's boundary data next to
    face f, laid out for the halo of the opposite face of the neighbour
    across f; recv[f]: this rank's halo buffer of face f.  Per dimension,
    first every rank sends across its high face and receives into its low
    halo, then the reverse; each phase's operations are posted together and
    waited for.  A neighbour that is this rank is served by a copy."""
    import torch.distributed as dist
    for d in dims:
        for up in (True, False):
            f_send = 2 * d + (1 if up else 0)
            f_recv = 2 * d + (0 if up else 1)
            to, frm = dec.neighbour(rank, f_send), dec.neighbour(rank, f_recv)
            ops = []
            if to is not None:
                if to == rank:
                    recv[OPPOSITE[f_send]].copy_(send[f_send])
                else:
                    ops.append(dist.P2POp(dist.isend, send[f_send], to, group=group))
            if frm is not None and frm != rank:
                ops.append(dist.P2POp(dist.irecv, recv[f_recv], frm, group=group))
            if ops:
                for w in dist.batch_isend_irecv(ops):
                    w.wait()


class LocalBlocks:
    """Every block of a decomposed grid as its own context on the current
    GPU and stream.  ``step()`` is one Runge-Kutta step of all blocks; the
    result equals one context's ``mhd_step`` on the whole grid, bitwise."""

    def __init__(self, cfg: Config, dims, force_halo: bool = False):
        import torch
        self.cfg = cfg
        self.dec = Decomposition(cfg.n, dims, cfg.bc, force_halo)
        self.blocks = [MHD(self.dec.local_config(cfg, r)) for r in range(self.dec.nblocks)]
        self.halo = [[b.halo_buffer(f) if f in self.dec.halo_faces(r) else None
                      for f in range(6)] for r, b in enumerate(self.blocks)]
        self.nstage = 3 if cfg.rk_order == 3 else 2
        self.lam = torch.zeros(1, dtype=torch.int64, device="cuda")

    def set_state(self, U, kind: int = 0):
        """U: the global float64 CUDA tensor (9, nz, ny, nx)."""
        for r, b in enumerate(self.blocks):
            b.set_state(self.dec.scatter(U, r).contiguous(), kind=kind)

    def get_state(self):
        import torch
        nx, ny, nz = self.cfg.n
        out = torch.empty((9, nz, ny, nx), dtype=torch.float64, device="cuda")
        return self.dec.gather([b.get_state() for b in self.blocks], out)

    def step(self):
        self.lam.zero_()
        for b in self.blocks:
            b.lambda_max_into(self.lam)
        for b in self.blocks:
            b.step_begin(0.0, 0.0, self.lam)
        for _ in range(self.nstage):
            for r in range(len(self.blocks)):
                for f in self.dec.halo_faces(r):
                    nb = self.dec.neighbour(r, f)
                    self.blocks[nb].halo_pack(OPPOSITE[f], self.halo[r][f])
            for r, b in enumerate(self.blocks):
                b.step_stage(self.halo[r])


class DistributedBlock:
    """This rank's block of a decomposed grid, on the current GPU, with the
    other ranks' blocks reached through ``torch.distributed`` (NCCL for CUDA
    tensors): ``step()`` packs the halo faces, exchanges them, runs each stage,
    and reduces the wave speed with an allreduce(MAX)."""

    def __init__(self, cfg: Config, dims, rank: int, group=None, force_halo: bool = False):
        import torch
        self.cfg, self.rank, self.group = cfg, rank, group
        self.dec = Decomposition(cfg.n, dims, cfg.bc, force_halo)
        self.solver = MHD(self.dec.local_config(cfg, rank))
        faces = self.dec.halo_faces(rank)
        self.recv = {f: self.solver.halo_buffer(f) for f in faces}
        self.send = {f: self.solver.halo_buffer(f) for f in faces}
        self.nstage = 3 if cfg.rk_order == 3 else 2
        self.lam = torch.zeros(1, dtype=torch.int64, device="cuda")

    def step(self):
        import torch.distributed as dist
        s = self.solver
        self.lam.zero_()
        s.lambda_max_into(self.lam)
        dist.all_reduce(self.lam, op=dist.ReduceOp.MAX, group=self.group)
        s.step_begin(0.0, 0.0, self.lam)
        halo = [self.recv.get(f) for f in range(6)]
        for _ in range(self.nstage):
            for f, buf in self.send.items():
                s.halo_pack(f, buf)
            exchange(self.dec, self.rank, self.send, self.recv, self.group)
            s.step_stage(halo)

