"""Pins of the oracle's floor branches of cons->prim (step 2 of the stage,
Section 3.2; the paper gives no floors, the reading is absolute floors by
replacement, counted once per stage for every interior cell of the stage
input).  Each count is checked against the decisions recomputed in numpy
from the plain formulas on the oracle's own stage inputs, and the replaced
values against the floor constants."""
import numpy as np
import pytest

import oracle as orc
from paper_2510_24175_gb300.inputs import Problem
from tests.parity_util import floor_decisions, grid_of, oracle_floor_run

PRS = 7


def defects(bc=(0,) * 6, limiter=2, rk=2, n=(24, 16, 10)):
    return Problem("floor_defects", n, seed=7, bc=bc, rho_floor=1e-3, p_floor=1e-3,
                   limiter=limiter, rk_order=rk, params=dict(n_rho=4, n_p=4))


@pytest.mark.parametrize("bc,limiter,rk", [((0,) * 6, 2, 2), ((0, 0, 1, 1, 1, 1), 2, 2),
                                           ((0,) * 6, 3, 3)])
def test_floor_counts_equal_the_decisions_on_every_stage_input(bc, limiter, rk):
    pb = defects(bc, limiter, rk)
    r, (n_rho, n_p, _), margin = oracle_floor_run(pb, 2)
    assert np.isfinite(r.U).all()
    assert n_rho > 0 and n_p > 0
    assert r.floors == (n_rho, n_p)
    assert margin > 1e-3


def test_floors_replace_density_and_pressure_by_the_floor_values():
    pb = defects()
    U = orc.prim_to_cons(pb.prim(), pb.gamma)
    V, (n_rho, n_p) = orc.cons_to_prim(U, grid_of(pb))
    rho_low = U[0] < pb.rho_floor
    m2 = U[1] ** 2 + U[2] ** 2 + U[3] ** 2
    b2 = U[4] ** 2 + U[5] ** 2 + U[6] ** 2
    p = (pb.gamma - 1.0) * (U[PRS] - 0.5 * m2 / np.maximum(U[0], pb.rho_floor) - 0.5 * b2)
    assert n_rho == rho_low.sum() == 4 and n_p == (p < pb.p_floor).sum() == 4
    assert np.all(V[0][rho_low] == pb.rho_floor)
    assert np.all(V[PRS][p < pb.p_floor] == pb.p_floor)
    # velocity of a floored cell: momentum over the floored density
    np.testing.assert_array_equal(V[1][rho_low], U[1][rho_low] / pb.rho_floor)


def test_ghost_copies_of_a_floored_boundary_cell_are_not_counted():
    """One negative-pressure cell in the corner of an outflow box: its
    outflow ghost copies are converted too, but a stage counts it once."""
    pb = Problem("uniform", (8, 6, 4), bc=(1,) * 6, p_floor=1e-3,
                 params=dict(V0=(1.0, 0.1, 0.0, 0.0, 0.3, 0.2, 0.1, 1.0, 0.0)))
    V = pb.prim()
    V[PRS, 0, 0, 0] = -0.5
    U = orc.prim_to_cons(V, pb.gamma)
    g = grid_of(pb)
    _, cnt = orc.stage(U, g, 1e-4, 2.0, 1)
    assert cnt == (0, 1)
    c, _ = floor_decisions(U, pb)
    assert c[:2] == (0, 1)
