"""CPU checks of the C-ABI boundary: the library builds, loads without a GPU
and exports every function declared in include/mhd.h; the Python binding
exposes the same names; argument validation needs no device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mhd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(mhd_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2510_24175_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_six_core_entry_points():
    names = declared_functions()
    for n in ["mhd_create", "mhd_set_state", "mhd_step", "mhd_dt", "mhd_adjoint_step",
              "mhd_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(built_lib):
    for name in declared_functions():
        assert hasattr(built_lib, name), name


def test_binding_names_match_header():
    import paper_2510_24175_gb300 as m
    assert sorted(m.EXPORTED) == declared_functions()
    for name in declared_functions():
        if name not in ("mhd_set_stream", "mhd_step_info", "mhd_counters",
                        "mhd_conserved_sums", "mhd_last_error", "mhd_profile_enable",
                        "mhd_profile_read") and not name.startswith("mhd_ensemble"):
            assert callable(getattr(m, name)), name


def test_config_validation_without_gpu(built_lib):
    import paper_2510_24175_gb300 as m
    m.lib()
    cfg = m.mhd_config_default()
    assert cfg.gamma == pytest.approx(5 / 3) and cfg.limiter == m.MHD_LIM_MC
    cfg.n[0], cfg.n[1], cfg.n[2] = 64, 32, 16
    assert m.mhd_workspace_bytes(cfg) >= 2 * 9 * 64 * 32 * 16 * 8
    bad = m.mhd_config_default()
    bad.n[0], bad.n[1], bad.n[2] = 8, 1, 8  # inactive y with active z
    with pytest.raises(m.MHDError):
        m.mhd_workspace_bytes(bad)
    bad = m.mhd_config_default()
    bad.n[0] = 8
    bad.bc[0] = m.MHD_BC_OUTFLOW  # periodic on one side only
    with pytest.raises(m.MHDError):
        m.mhd_workspace_bytes(bad)
    bad = m.mhd_config_default()
    bad.n[0] = 8
    bad.gamma = 1.0
    with pytest.raises(m.MHDError):
        m.mhd_workspace_bytes(bad)
    fp32 = m.mhd_config_default()
    fp32.n[0] = 8
    fp32.precision = m.MHD_FP32
    fp32.flags = m.MHD_FLAG_ADJOINT
    with pytest.raises(m.MHDError):
        m.mhd_workspace_bytes(fp32)


def test_flux_batch_rejects_bad_arguments(built_lib):
    import paper_2510_24175_gb300 as m
    L = m.lib()
    assert L.mhd_flux_batch(None, None, None, 10, 0, 1.0, 5 / 3, 0, None) == m.MHD_ERR_INVALID


def test_fma_rate_probe_rejects_a_null_output(built_lib):
    import paper_2510_24175_gb300 as m
    L = m.lib()
    assert L.mhd_fp64_fma_rate(None, 0xFF, None) == m.MHD_ERR_INVALID
    assert L.mhd_last_error(None) == b"mhd_fp64_fma_rate: out is NULL"


def test_context_free_failures_leave_a_message(built_lib):
    """Calls without a context (configuration checks, flux batch, ensemble
    sizing) leave the reason of a failure for mhd_last_error(NULL), per host
    thread; the binding puts it into the raised error."""
    import ctypes
    import threading
    import paper_2510_24175_gb300 as m
    L = m.lib()
    cfg = m.mhd_config_default()
    cfg.n[0], cfg.n[1], cfg.n[2] = 8, 1, 8
    with pytest.raises(m.MHDError) as e:
        m.mhd_workspace_bytes(cfg)
    assert "ny = 1 needs nz = 1" in str(e.value)
    cfg = m.mhd_config_default()
    cfg.n[0] = 8
    cfg.cfl = 1.5
    with pytest.raises(m.MHDError) as e:
        m.mhd_workspace_bytes(cfg)
    assert "cfl" in str(e.value)
    assert L.mhd_flux_batch(None, None, None, 10, 0, 1.0, 5 / 3, 0, None) == m.MHD_ERR_INVALID
    assert L.mhd_last_error(None) == b"mhd_flux_batch: bad argument"
    # ensemble: box 1 is FP64, which the batched kernel does not take
    boxes = (m.mhd_config * 2)()
    for b in range(2):
        boxes[b] = m.mhd_config_default()
        boxes[b].n[0] = boxes[b].n[1] = boxes[b].n[2] = 16
        boxes[b].precision = m.MHD_FP32
    boxes[1].precision = m.MHD_FP64
    nb = ctypes.c_size_t(0)
    assert L.mhd_ensemble_workspace_bytes(boxes, 2, ctypes.byref(nb)) == m.MHD_ERR_INVALID
    assert L.mhd_last_error(None).startswith(b"ensemble box 1:")
    boxes[1].precision = m.MHD_FP32
    boxes[1].n[0] = 1
    assert L.mhd_ensemble_workspace_bytes(boxes, 2, ctypes.byref(nb)) == m.MHD_ERR_INVALID
    assert L.mhd_last_error(None) == b"ensemble box 1: invalid config: x must be active (nx >= 2)"
    # another thread keeps its own message
    seen = []
    t = threading.Thread(target=lambda: seen.append(L.mhd_last_error(None)))
    t.start()
    t.join()
    assert seen == [b"no error"]
    assert L.mhd_last_error(None) == b"ensemble box 1: invalid config: x must be active (nx >= 2)"


def _paper_configs():
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_benchmark_configs.txt")
    rows = []
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            name, grid, rec, rk, divb, prec, _ = [f.strip() for f in line.split("|")]
            rows.append((name, tuple(int(x) for x in grid.split()), rec, rk, divb, prec))
    return rows


def test_paper_benchmark_configs_are_accepted(built_lib):
    """The paper's stated gPLUTO benchmark configurations (Section 4.2;
    tests/golden/paper_benchmark_configs.txt) are valid configurations of the
    library, and its memory statement holds for this layout: divergence
    cleaning needs less device memory than constrained transport, which let
    the strong-scaling runs take a slightly larger grid (832^2 x 416 with GLM
    needs no more than 704^2 x 352 with CT).  The per-node grids of both fit
    one GB300 (284,208 MiB)."""
    import paper_2510_24175_gb300 as m
    m.lib()
    rows = _paper_configs()
    assert len(rows) == 4
    need = {}
    for name, n, rec, rk, divb, prec in rows:
        cfg = m.mhd_config_default()
        cfg.n[0], cfg.n[1], cfg.n[2] = n
        cfg.limiter = {"WENOZ": m.MHD_LIM_WENOZ}[rec]
        cfg.rk_order = {"RK3": 3}[rk]
        cfg.divb = {"CT": m.MHD_DIVB_CT, "GLM": m.MHD_DIVB_GLM}[divb]
        cfg.precision = {"FP64": m.MHD_FP64}[prec]
        need[name] = m.mhd_workspace_bytes(cfg)
        cfg.divb = m.MHD_DIVB_GLM if cfg.divb == m.MHD_DIVB_CT else m.MHD_DIVB_CT
        other = m.mhd_workspace_bytes(cfg)
        glm, ct = (need[name], other) if divb == "GLM" else (other, need[name])
        assert glm < ct, name
    assert need["strong_scaling_group1_base"] <= need["orszag_tang_weak_scaling_per_node"]
    gb300 = 284208 * 2 ** 20
    assert need["orszag_tang_weak_scaling_per_node"] < gb300
    assert need["strong_scaling_group1_base"] < gb300
