"""Batched ensemble (one persistent, cooperative, graph-captured launch for
all boxes) against per-box plain launches: every box must be bitwise equal
to the same box advanced alone with mhd_step, across several step calls and
after the autotuner has changed the work decomposition."""
import numpy as np
import pytest

from paper_2510_24175_gb300 import inputs

pytestmark = pytest.mark.gpu


def _boxes(sizes, seed=5):
    rng = np.random.default_rng(seed)
    b0s = rng.uniform(0.1, 0.5, size=len(sizes))
    pbs = []
    for n, b0 in zip(sizes, b0s):
        pb = inputs.orszag_tang_3d(int(n))
        pb.params = {"B0": float(b0)}
        pb.precision = 1
        pbs.append(pb)
    return pbs


def _run_pair(pbs, step_calls, autotune=False, tiles=None):
    import torch
    import paper_2510_24175_gb300 as m
    cfgs = [m.Config.from_problem(pb) for pb in pbs]
    ens = m.Ensemble(cfgs)
    plain = [m.MHD(c) for c in cfgs]
    for b, pb in enumerate(pbs):
        V = torch.from_numpy(pb.prim()).cuda()
        ens.set_state(b, V, kind=m.MHD_PRIM)
        plain[b].set_state(V, kind=m.MHD_PRIM)
    if autotune:
        ens.autotune(1)
    for b, (ty, tz) in (tiles or {}).items():
        ens.set_tiles(b, ty, tz)
    total = 0
    for k in step_calls:
        ens.step(k)
        total += k
    for s in plain:
        for _ in range(total):
            s.step()
    return ens, plain, total


def test_ensemble_bitwise_equals_per_box_launches():
    pbs = _boxes([16, 24, 32, 16, 40, 24])
    ens, plain, total = _run_pair(pbs, [2, 1])
    for b in range(len(pbs)):
        a = ens.get_state(b)
        r = plain[b].get_state()
        assert bool((a == r).all()), f"box {b} differs"
        ie, ip = ens.info(b), plain[b].step_info()
        assert ie["t"] == ip["t"] and ie["steps"] == total and ie["dt"] == ip["dt"]


def test_ensemble_after_autotune_and_graph_reuse():
    pbs = _boxes([32, 48, 16, 32], seed=6)
    ens, plain, total = _run_pair(pbs, [1, 1, 2], autotune=True)
    for b in range(len(pbs)):
        assert bool((ens.get_state(b) == plain[b].get_state()).all()), f"box {b} differs"
    info = ens.info(0)
    assert info["graph"] and info["tz"] in (4, 8, 16, 32) and info["ty"] in (4, 8)


@pytest.mark.parametrize("ty", [4, 8])
def test_ensemble_tile_shapes_bitwise_equal_to_plain_launches(ty):
    """The persistent launch on 32 x ty column tiles with ragged rows and odd
    z-chunk depths: each box bitwise equal to its own per-box launches
    (which run 32 x 8 tiles and the context's own z chunks)."""
    pbs = _boxes([32, 48, 16, 33], seed=7)
    tiles = {0: (ty, 5), 1: (ty, 48), 2: (ty, 3), 3: (ty, 1)}
    ens, plain, total = _run_pair(pbs, [1, 2], tiles=tiles)
    for b in range(len(pbs)):
        assert bool((ens.get_state(b) == plain[b].get_state()).all()), f"box {b} differs"
        inf = ens.info(b)
        assert (inf["ty"], inf["tz"]) == (tiles[b][0], min(tiles[b][1], pbs[b].n[2]))


def test_ensemble_rejects_fp64_and_2d_boxes():
    import paper_2510_24175_gb300 as m
    with pytest.raises(m.MHDError):
        m.Ensemble([m.Config(n=(16, 16, 16), precision=m.MHD_FP64)])
    with pytest.raises(m.MHDError):
        m.Ensemble([m.Config(n=(16, 16, 1), precision=m.MHD_FP32)])
