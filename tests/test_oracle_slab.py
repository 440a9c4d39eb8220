"""The slab-parallel oracle runner (oracle/slab.py: the oracle on all host
cores, z slabs exchanging ghost planes through shared memory, the paper's
boundary exchange between subdomains, Section 3.2) is bitwise the
undecomposed oracle run, for both schemes and both z boundary rules."""
import numpy as np
import pytest

import oracle as orc
from oracle.slab import SlabRunner, _slabs
from paper_2510_24175_gb300.inputs import Problem
from tests.parity_util import grid_of


def test_slabs_cover_the_grid():
    for nz, p in [(256, 16), (17, 4), (12, 5), (3, 1)]:
        s = _slabs(nz, p)
        assert s[0][0] == 0 and s[-1][1] == nz
        assert all(a[1] == b[0] for a, b in zip(s, s[1:]))
        assert max(h - l for l, h in s) - min(h - l for l, h in s) <= 1


@pytest.mark.parametrize("lim,rk,bc", [(2, 2, (0,) * 6), (2, 2, (0, 0, 1, 1, 1, 1)),
                                       (3, 3, (0,) * 6)])
def test_slab_runner_is_bitwise_the_oracle_run(lim, rk, bc):
    pb = Problem("random_smooth", (14, 10, 19), seed=23, limiter=lim, rk_order=rk, bc=bc)
    g = grid_of(pb)
    U0 = orc.prim_to_cons(pb.prim(), pb.gamma)
    ref = orc.run(U0, g, 3)
    with SlabRunner(g, nproc=4) as r:
        got = r.run(U0, 3)
        # a second run on the same pool starts afresh
        got2 = r.run(U0, 2)
        dt_ch = r.cfl_dt(got.U)
    np.testing.assert_array_equal(got.U, ref.U)
    np.testing.assert_array_equal(got.dts, ref.dts)
    np.testing.assert_array_equal(got.chs, ref.chs)
    assert got.t == ref.t
    np.testing.assert_array_equal(got2.U, orc.run(U0, g, 2).U)
    assert dt_ch == orc.cfl_dt(ref.U, g)
