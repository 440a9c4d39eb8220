"""Shared helpers of the parity tests: problem -> oracle grid, GPU runs through
the C ABI, the relative-L1 norm, and the oracle's one-step value at sampled
cells of a large periodic grid (a local sub-box computation)."""
import numpy as np

import oracle as orc
from paper_2510_24175_gb300.inputs import Problem

RHO, VX, VY, VZ, BX, BY, BZ, PRS, PSI = range(9)


def grid_of(pb: Problem) -> orc.Grid:
    return orc.Grid(n=pb.n, dx=pb.dx, gamma=pb.gamma, glm_alpha=pb.glm_alpha,
                    rho_floor=pb.rho_floor, p_floor=pb.p_floor, limiter=pb.limiter,
                    bc=pb.bc, cfl=pb.cfl, rk_order=pb.rk_order)


def rel_l1(a: np.ndarray, b: np.ndarray, floor: float = 1e-3) -> np.ndarray:
    """Per variable ||a-b||_1 / max(||b||_1, floor ||rho_b||_1): the floor keeps
    near-zero planes (psi, a vanishing component) from dividing by ~0.  FP32
    comparisons use floor = 0.1, since there psi and components that start at
    zero carry FP32 round-off noise of absolute size ~1e-7 of the field."""
    num = np.abs(a - b).reshape(9, -1).sum(axis=1)
    den = np.abs(b).reshape(9, -1).sum(axis=1)
    den = np.maximum(den, floor * den[RHO])
    return num / den


def oracle_run(pb: Problem, nsteps: int, t_end: float = 0.0):
    g = grid_of(pb)
    U0 = orc.prim_to_cons(pb.prim(), pb.gamma)
    if getattr(pb, "divb", 0) == 1:
        return orc.ct_run(U0, pb.faces(), g, nsteps, t_end=t_end)
    return orc.run(U0, g, nsteps, t_end=t_end)


def gpu_run(pb: Problem, nsteps: int, precision=None, record=False):
    """Runs nsteps CFL steps through the C ABI (device computes dt); returns
    (U as numpy float64, list of (t, dt, ch) per step when record)."""
    import torch
    import paper_2510_24175_gb300 as m
    cfg = m.Config.from_problem(pb, precision=precision)
    s = m.MHD(cfg)
    s.set_state(torch.from_numpy(pb.prim()).cuda(), kind=m.MHD_PRIM)
    if getattr(pb, "divb", 0) == m.MHD_DIVB_CT:
        s.set_face_field(torch.from_numpy(pb.faces()).cuda())
    hist = []
    for _ in range(nsteps):
        s.step()
        if record or pb.t_end > 0:
            info = s.step_info()
            hist.append((info["t"], info["dt"], info["ch"]))
            if pb.t_end > 0 and info["t"] >= pb.t_end:
                break
    U = s.get_state().cpu().numpy()
    counters = s.counters()
    return U, hist, counters


def sampled_one_step(U0: np.ndarray, pb: Problem, dt: float, ch: float, cells, radius=None,
                     faces=None):
    """Oracle value after one step at the given (k, j, i) cells of a fully
    periodic grid, for the problem's reconstruction and Runge-Kutta order
    (and constrained transport when `faces`, the face field, is given).  A
    cell's new value depends only on cells within `radius` along each axis
    (stages x ghost depth, plus two cells per stage for constrained
    transport's edge fields and face means, plus one spare), so the oracle advances a
    (2 radius + 1)^3 box cut out around the cell (periodic wrap) with the
    global dt and c_h and reads its centre; the box's own boundary treatment
    cannot reach the centre."""
    rk = getattr(pb, "rk_order", 2)
    ghost = 3 if pb.limiter == orc.LIM_WENOZ else 2
    if radius is None:
        radius = rk * (ghost + (2 if faces is not None else 0)) + (1 if rk != 2 or faces is not None else 0)
    out = np.empty((9, len(cells)))
    w = 2 * radius + 1
    sub = Problem(pb.name, (w, w, w), xmin=(0, 0, 0),
                  xmax=(w * pb.dx[0], w * pb.dx[1], w * pb.dx[2]), gamma=pb.gamma,
                  limiter=pb.limiter, glm_alpha=pb.glm_alpha, rho_floor=pb.rho_floor,
                  p_floor=pb.p_floor, bc=(1,) * 6 if faces is None else (0,) * 6,
                  rk_order=rk)
    g = grid_of(sub)
    nz, ny, nx = U0.shape[1:]
    for m, (k, j, i) in enumerate(cells):
        kk = np.arange(k - radius, k + radius + 1) % nz
        jj = np.arange(j - radius, j + radius + 1) % ny
        ii = np.arange(i - radius, i + radius + 1) % nx
        box = np.ascontiguousarray(U0[:, kk][:, :, jj][:, :, :, ii])
        if faces is None:
            r = orc.run(box, g, 1, dts=[dt], chs=[ch])
        else:
            fbox = np.ascontiguousarray(faces[:, kk][:, :, jj][:, :, :, ii])
            r = orc.ct_run(box, fbox, g, 1, dts=[dt], chs=[ch])
        out[:, m] = r.U[:, radius, radius, radius]
    return out


def floor_decisions(W: np.ndarray, pb: Problem):
    """The decisions the conversion of a stage input W takes at each interior
    cell, from the plain formulas in FP64: (rho floored, p floored, FP32
    pressure recomputed in FP64), and the smallest relative distance of any
    of them from its threshold.  Density first; the pressure uses the
    floored density.  The FP32 path recomputes p in FP64 when p < p_floor or
    p < 1e-3 (gamma - 1) E, and floors it when the FP64 value is below
    p_floor.  A decision farther than about 1e-3 from its threshold is taken
    alike by the FP64 oracle and by either GPU precision."""
    rho = W[RHO]
    rho_f = rho < pb.rho_floor
    r = np.where(rho_f, pb.rho_floor, rho)
    kin = 0.5 * (W[VX] ** 2 + W[VY] ** 2 + W[VZ] ** 2) / r
    mag = 0.5 * (W[BX] ** 2 + W[BY] ** 2 + W[BZ] ** 2)
    p = (pb.gamma - 1.0) * (W[PRS] - kin - mag)
    p_f = p < pb.p_floor
    cold = p < 1e-3 * (pb.gamma - 1.0) * W[PRS]
    branch = p_f | cold

    def margin(a, t):
        t = np.broadcast_to(np.asarray(t, dtype=np.float64), a.shape)
        with np.errstate(divide="ignore", invalid="ignore"):
            m = np.where(t > 0, np.abs(a / t - 1.0), np.inf)
        return np.where(np.isfinite(m), m, np.inf)

    m = min(float(margin(rho, pb.rho_floor).min()), float(margin(p, pb.p_floor).min()),
            float(margin(p, 1e-3 * (pb.gamma - 1.0) * W[PRS]).min()))
    return (int(rho_f.sum()), int(p_f.sum()), int(branch.sum())), m


def oracle_floor_run(pb: Problem, nsteps: int):
    """Oracle run of nsteps CFL steps with the decision counts of every
    stage input (floor_decisions of U^n and of the first stage U1, and of
    U2 with SSP-RK3): returns (RunResult, counts (rho, p, branch), margin)."""
    g = grid_of(pb)
    U0 = orc.prim_to_cons(pb.prim(), pb.gamma)
    U = U0
    tot = np.zeros(3, dtype=np.int64)
    margin = np.inf
    for _ in range(nsteps):
        dt, ch = orc.cfl_dt(U, g)
        inputs = [U]
        U1, _ = orc.stage(U, g, dt, ch, 1)
        inputs.append(U1)
        if g.rk_order == 3:
            U2, _ = orc.stage(U1, g, dt, ch, 2, Un=U)
            inputs.append(U2)
        for W in inputs:
            c, m = floor_decisions(W, pb)
            tot += c
            margin = min(margin, m)
        U = orc.run(U, g, 1).U
    return orc.run(U0, g, nsteps), tuple(int(x) for x in tot), margin
