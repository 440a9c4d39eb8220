"""mhd_conserved_sums_noalloc: the entry point for callers that can't
allocate device memory (their GPU memory belongs to another allocator, their
policy forbids allocations inside the time loop, or they are capturing a
stream).  Called through the C ABI, it must give the same conservation sums
as the context-based mhd_conserved_sums, on two calls in a row (the shared
internal scratch keeps the previous call's contents), and reject grids larger
than its fixed scratch.  Collected last so a stop-at-first-failure run has run
every other test first."""
import ctypes

import numpy as np
import pytest

import oracle as orc
from paper_2510_24175_gb300.inputs import Problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_sums_match_context_sums_twice(precision):
    import torch
    import paper_2510_24175_gb300 as m
    pb = Problem("random_smooth", (70, 33, 21), seed=21)
    U64 = orc.prim_to_cons(pb.prim(), pb.gamma)
    cfg = m.Config.from_problem(pb, precision=precision)
    s = m.MHD(cfg)
    s.set_state(torch.from_numpy(U64).cuda())
    ref = s.conserved_sums()
    # the caller's own state array in the context's precision
    U = torch.from_numpy(U64).cuda()
    if precision == 1:
        U = U.float()
    c = cfg.c()
    L = m.lib()
    for _ in range(2):
        out = (ctypes.c_double * 8)()
        rc = L.mhd_conserved_sums_noalloc(ctypes.byref(c), ctypes.c_void_p(U.data_ptr()), out,
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == m.MHD_OK
        got = np.array(out[:])
        scale = np.abs(ref).max()
        np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13 * scale)


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    import paper_2510_24175_gb300 as m
    cfg = m.Config(n=(1024, 1024, 1024)).c()  # 2^30 cells > 16384 * 32768
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = (ctypes.c_double * 8)()
    rc = m.lib().mhd_conserved_sums_noalloc(ctypes.byref(cfg), ctypes.c_void_p(dummy.data_ptr()),
                                            out, None)
    assert rc == m.MHD_ERR_NOMEM


def test_noalloc_refuses_a_capturing_stream_and_leaves_the_capture_intact():
    """The call ends with a host copy and a stream synchronisation, which a
    capturing stream does not accept: it must refuse such a stream before it
    enqueues anything, so the caller's capture can still be completed."""
    import torch
    import paper_2510_24175_gb300 as m
    pb = Problem("random_smooth", (40, 20, 12), seed=5)
    U = torch.from_numpy(orc.prim_to_cons(pb.prim(), pb.gamma)).cuda()
    c = m.Config.from_problem(pb).c()
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            out = (ctypes.c_double * 8)()
            rc = m.lib().mhd_conserved_sums_noalloc(
                ctypes.byref(c), ctypes.c_void_p(U.data_ptr()), out,
                ctypes.c_void_p(s.cuda_stream))
            y.add_(1.0)
    assert rc == m.MHD_ERR_INVALID
    assert b"capturing" in m.lib().mhd_last_error(None)
    g.replay()
    torch.cuda.synchronize()
    assert float(y.sum()) == 8.0
    # and the entry point still works afterwards on an ordinary stream
    got = m.mhd_conserved_sums_noalloc(m.Config.from_problem(pb).c(), U)
    assert np.isfinite(got).all()
