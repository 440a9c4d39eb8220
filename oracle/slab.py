"""The oracle advanced on all host cores by z slabs -- test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may use this module.  It runs the oracle as it stands: each worker
process (started with ``spawn``) owns a slab of z planes of a grid whose full
state lives in shared memory, and per step

  1. computes the maximum wave speed of its slab (``orc_max_speed``); the
     global maximum is exact, so c_h = lambda and dt = cfl / (c_h sum 1/dx_d)
     are the undecomposed run's;
  2. per Runge-Kutta stage, builds its padded slab from the shared stage
     input -- ghost zones in x and y by the boundary rule, z ghost planes from
     the neighbouring slabs or by the boundary rule at the ends: the paper's
     boundary exchange between subdomains (Section 3.2) -- and calls the
     oracle's stage on it (``orc_stage_padded``), writing its slab of the
     stage output.

The result is bitwise that of ``oracle.run`` on the whole grid (the per-cell
arithmetic is identical once the ghost values are).  Floor activations are
not counted here.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

from . import Grid, RunResult

_MODE = {0: "wrap", 1: "edge"}  # periodic, outflow


def _slabs(nz: int, nproc: int):
    """[z_lo, z_hi) of each worker: contiguous, as even as possible."""
    base, extra = divmod(nz, nproc)
    out, z = [], 0
    for r in range(nproc):
        h = base + (1 if r < extra else 0)
        out.append((z, z + h))
        z += h
    return out


def _padded(W: np.ndarray, z0: int, z1: int, grid: Grid) -> np.ndarray:
    """Slab [z0, z1) of W with its ghost zones filled by the boundary rules
    (ghost width 2 for PLM, 3 for WENO-Z, in active dimensions)."""
    nx, ny, nz = grid.n
    g = [grid.ghost if n > 1 else 0 for n in grid.n]
    kk = np.arange(z0 - g[2], z1 + g[2])
    kk = kk % nz if grid.bc[4] == 0 else np.clip(kk, 0, nz - 1)
    P = W[:, kk]
    if g[0]:
        P = np.pad(P, [(0, 0), (0, 0), (0, 0), (g[0], g[0])], mode=_MODE[grid.bc[0]])
    if g[1]:
        P = np.pad(P, [(0, 0), (0, 0), (g[1], g[1]), (0, 0)], mode=_MODE[grid.bc[2]])
    return np.ascontiguousarray(P)


def _worker(rank, nproc, names, shape, grid_kw, conn):
    """Serves the parent's commands on conn: ("lam",) -> the slab's maximum
    wave speed; ("stage", s, dt, ch) -> stage s of the step on the slab;
    ("stop",)."""
    import oracle as orc
    shms = [shared_memory.SharedMemory(name=n) for n in names]
    try:
        A, B, C = (np.ndarray(shape, dtype=np.float64, buffer=s.buf) for s in shms)
        grid = Grid(**grid_kw)
        z0, z1 = _slabs(grid.n[2], nproc)[rank]
        local = Grid(**{**grid_kw, "n": (grid.n[0], grid.n[1], z1 - z0)})
        Un = None
        while True:
            cmd = conn.recv()
            if cmd[0] == "stop":
                return
            if cmd[0] == "lam":
                conn.send(orc.max_speed(np.ascontiguousarray(A[:, z0:z1]), local))
                continue
            _, st, dt, ch = cmd
            last = st == grid.rk_order
            if st == 1:
                Un = np.ascontiguousarray(A[:, z0:z1])
                B[:, z0:z1] = orc.stage_padded(_padded(A, z0, z1, grid), local, dt, ch, 1)
            elif not last:  # the middle stage of SSP-RK3
                C[:, z0:z1] = orc.stage_padded(_padded(B, z0, z1, grid), local, dt, ch, 2, Un=Un)
            else:
                W = C if grid.rk_order == 3 else B
                A[:, z0:z1] = orc.stage_padded(_padded(W, z0, z1, grid), local, dt, ch, st,
                                               Un=Un, damp=True)
            conn.send(True)
    finally:
        for s in shms:
            s.close()


class SlabRunner:
    """A pool of ``nproc`` slab workers for one grid (z must be active, with
    at least ghost-width planes per slab).  Use as a context manager.  A
    worker that dies or raises makes the running call raise (nothing waits
    for it)."""

    def __init__(self, grid: Grid, nproc: int | None = None, timeout: float = 3600.0):
        from dataclasses import asdict
        nproc = nproc or os.cpu_count() or 1
        nproc = max(1, min(nproc, grid.n[2] // grid.ghost))
        self.grid, self.nproc, self.timeout = grid, nproc, timeout
        nx, ny, nz = grid.n
        self.shape = (9, nz, ny, nx)
        nbytes = 9 * nx * ny * nz * 8
        self._shm = [shared_memory.SharedMemory(create=True, size=nbytes) for _ in range(3)]
        self.A = np.ndarray(self.shape, dtype=np.float64, buffer=self._shm[0].buf)
        ctx = mp.get_context("spawn")
        kw = asdict(grid)
        names = [s.name for s in self._shm]
        self._conns, self._procs = [], []
        for r in range(nproc):
            parent, child = ctx.Pipe()
            p = ctx.Process(target=_worker, args=(r, nproc, names, self.shape, kw, child),
                            daemon=True)
            p.start()
            child.close()
            self._conns.append(parent)
            self._procs.append(p)
        self._open = True

    def _all(self, cmd):
        """Sends cmd to every worker and returns their replies in rank order;
        raises if a worker exits or does not answer within the timeout."""
        from multiprocessing.connection import wait
        for c in self._conns:
            c.send(cmd)
        out = [None] * self.nproc
        pending = dict(enumerate(self._conns))
        sentinels = {p.sentinel: r for r, p in enumerate(self._procs)}
        while pending:
            ready = wait(list(pending.values()) + list(sentinels), timeout=self.timeout)
            if not ready:
                raise TimeoutError(f"slab workers did not answer {cmd[0]!r} in {self.timeout} s")
            for obj in ready:
                if obj in sentinels and sentinels[obj] in pending:
                    raise RuntimeError(f"slab worker {sentinels[obj]} exited")
                for r, c in list(pending.items()):
                    if c is obj:
                        try:
                            out[r] = c.recv()
                        except EOFError:
                            raise RuntimeError(f"slab worker {r} exited") from None
                        del pending[r]
        return out

    def _lambda(self) -> float:
        ch = 0.0
        for v in self._all(("lam",)):  # NaN-sticky maximum, as the oracle's
            if not (v <= ch):
                ch = float(v)
        return ch

    def cfl_dt(self, U: np.ndarray):
        """(dt, c_h) of the CFL rule for state U, as ``oracle.cfl_dt``."""
        self.A[...] = U
        ch = self._lambda()
        inv = sum(1.0 / self.grid.dx[d] for d in range(3) if self.grid.n[d] > 1)
        return self.grid.cfl / (ch * inv), ch

    def run(self, U0: np.ndarray, nsteps: int, t0: float = 0.0, dts=None,
            chs=None) -> RunResult:
        """nsteps steps from U0 (CFL rule, or the given dt / c_h sequences);
        the same result as ``oracle.run(U0, grid, nsteps)``."""
        grid = self.grid
        self.A[...] = U0
        inv = sum(1.0 / grid.dx[d] for d in range(3) if grid.n[d] > 1)
        out_dt, out_ch = np.zeros(nsteps), np.zeros(nsteps)
        t = t0
        for s in range(nsteps):
            if dts is not None and dts[s] > 0.0:
                dt, ch = float(dts[s]), float(chs[s])
            else:
                ch = self._lambda()
                dt = grid.cfl / (ch * inv)
            for st in range(1, grid.rk_order + 1):
                self._all(("stage", st, dt, ch))
            out_dt[s], out_ch[s] = dt, ch
            t += dt
        return RunResult(self.A.copy(), t, out_dt, out_ch)

    def close(self):
        if not self._open:
            return
        self._open = False
        for c in self._conns:
            try:
                c.send(("stop",))
            except Exception:
                pass
        for p in self._procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
        for c in self._conns:
            c.close()
        for s in self._shm:
            s.close()
            s.unlink()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
