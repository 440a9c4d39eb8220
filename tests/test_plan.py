"""Host-only launch planning of the 3-D stage kernels (mhd_plan_z_chunks,
no GPU): the z-chunk depth against a plain list-scheduling simulation of the
launch written here (every CTA pushed through a heap of slot free times),
the lower bounds any schedule obeys, and the depths of the bench workloads'
launches (the grid z extents of those launches in the ncu launch list)."""
import heapq
import math
import random

import pytest

import paper_2510_24175_gb300 as m

CANDIDATES = [256, 192, 128, 96, 80, 64, 56, 48, 40, 32, 24, 20, 16, 12, 8, 4]


def simulate(cols, nz, tz, slots):
    """Duration of one launch: CTAs in launch order (all full chunks of every
    column tile, then every column tile's last chunk), each on the slot that
    frees first, a CTA costing its planes plus one."""
    chunks = [min(tz, nz - z0) for z0 in range(0, nz, tz)]
    order = [c for c in chunks[:-1] for _ in range(cols)] + [chunks[-1]] * cols
    free = [0.0] * slots
    end = 0.0
    for planes in order:
        t = heapq.heappop(free) + planes + 1.0
        heapq.heappush(free, t)
        end = max(end, t)
    return end


def best_depth(cols, nz, slots):
    best, best_span = None, math.inf
    for tz in CANDIDATES:  # deepest first: a tie keeps the deeper chunk
        if tz > nz and tz != 4:
            continue
        sp = simulate(cols, nz, tz, slots)
        if sp < best_span:
            best, best_span = tz, sp
    return best, best_span


def cols_of(n, ty):
    return ((n[0] + 31) // 32) * ((n[1] + ty - 1) // ty)


@pytest.mark.parametrize("n,ty,per_sm,tz", [
    ((256, 256, 256), 8, 1, 48),   # FP64 PLM, Orszag-Tang 256^3: grid (8, 32, 6)
    ((512, 512, 512), 8, 2, 96),   # FP32 PLM, turbulent 512^3: grid (16, 64, 6)
    ((512, 512, 512), 8, 1, 128),  # FP64 PLM, turbulent 512^3: grid (16, 64, 4)
    ((256, 256, 256), 8, 2, 32),   # FP32 PLM, Orszag-Tang 256^3: grid (8, 32, 8)
    ((256, 256, 256), 4, 1, 48),   # FP64 WENO-Z, Orszag-Tang 256^3: grid (8, 64, 6)
])
def test_bench_workload_depths(n, ty, per_sm, tz):
    got, span = m.mhd_plan_z_chunks(n, ty, 152, per_sm)
    assert got == tz
    assert span == simulate(cols_of(n, ty), n[2], tz, 152 * per_sm)


def test_depth_is_the_shortest_simulated_launch():
    rng = random.Random(7)
    for _ in range(40):
        n = (rng.choice([32, 48, 64, 96, 128, 160, 200, 256]),
             rng.choice([8, 24, 64, 100, 128, 256]),
             rng.randint(2, 300))
        ty = rng.choice([4, 8])
        nsm, per_sm = rng.choice([(152, 1), (152, 2), (20, 1), (7, 3)])
        tz, span = m.mhd_plan_z_chunks(n, ty, nsm, per_sm)
        cols, slots = cols_of(n, ty), nsm * per_sm
        want_tz, want_span = best_depth(cols, n[2], slots)
        assert (tz, span) == (want_tz, want_span), (n, ty, nsm, per_sm)
        # any schedule: at least the work spread over every slot, and at
        # least the longest CTA
        chunks = [min(tz, n[2] - z0) for z0 in range(0, n[2], tz)]
        work = cols * sum(c + 1.0 for c in chunks)
        assert span >= work / slots - 1e-9
        assert span >= max(chunks) + 1.0


def test_grids_that_are_not_3d_take_one_plane_per_cta():
    assert m.mhd_plan_z_chunks((1024, 1, 1), 1, 152, 1)[0] == 1
    assert m.mhd_plan_z_chunks((512, 512, 1), 8, 152, 1)[0] == 1


def test_bad_arguments_are_rejected():
    for args in [((0, 8, 8), 8, 152, 1), ((8, 8, 8), 0, 152, 1), ((8, 8, 8), 8, 0, 1),
                 ((8, 8, 8), 8, 152, 0)]:
        with pytest.raises(m.MHDError):
            m.mhd_plan_z_chunks(*args)
