#!/usr/bin/env python
"""Benchmark of the GLM-MHD RK2 hot path on GB300.

Workload (one GPU): 3-D Orszag-Tang vortex, 256^3 periodic, FP64, MC limiter,
HLLD + GLM, RK2, CFL 0.8.  A bench step is one full RK2 step of the whole
grid (ghost remap, cons->prim, PLM, GLM + HLLD, flux divergence, both RK
stages, GLM damping, the max-wave-speed reduction and the device-side dt).
Metric: zone-updates/s = interior cells x steps / time.  The state (1.2 GB
per array) is far larger than L2 (129 MB), so no flush is needed between
steps.

Also reported on the same line: the FP32-bulk sweep (turbulent box 512^3)
and FP64 on that grid and on the FP64 workload's grid (same-grid precision
ratios), per-kernel CUDA-event times, roofline fractions against
MEASURED_PEAKS.json, end-to-end throughput through the C ABI with pinned host
buffers, the paper's WENO-Z + SSP-RK3 schemes (GLM and constrained
transport), the adjoint/forward step-time ratio, the batched ensemble, the
1-D Brio-Wu run to t = 0.1 as GPU wall time, SM clocks sampled during the
timed region, and the CPU oracle timed on the host cores.

--impl reference times the CPU FP64 oracle (there is no runnable reference
code for this paper) on bounded samples of the same workload.

N > 1 ranks (torchrun): every rank advances its own replica of the workload
(independent problems, no data-path collective); value = all zone-updates
over the max time across ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP64-pipe lane-instructions (DADD, DMUL, DFMA, DSETP, DMNMX, conversions)
# per cell executed by the FP64 stage kernel, stage 1 and stage 2 (which adds
# the GLM damping and the FP32 estimates of the next step's wave speed): ncu
# smsp__inst_executed_pipe_fp64 x 32 / cells over the timed steps of this
# bench's Orszag-Tang 256^3 run (profiles/).  They change whenever the kernel
# does.
FP64_INST_PER_CELL = {1: 1183.0, 2: 1211.0}
# DRAM bytes per cell of the stage kernel's launches (ncu dram__bytes_read +
# dram__bytes_write over the timed steps of this bench's 256^3 FP64 and 512^3
# FP32 runs, profiles/); reported as the roofline's traffic per launch.  Set
# to None whenever the kernel changes until they are captured again.
TRAFFIC_BYTES_PER_CELL = {8: {1: 151.9, 2: 224.4}, 4: {1: 75.65, 2: 111.64}}
# Nominal FP64 peak: 2 lanes/clk/SM x 152 SMs x 2.07 GHz = 629 G
# lane-instructions/s (1.26 TFLOP/s counting an FMA as 2).  The measured one,
# mhd_fp64_fma_rate in the same run, is reported beside it (about 1.68
# lanes/clk/SM: the SM's FP64 unit is shared by its warps, and one warp issues
# an FP64 instruction at most every 64 clocks).
FP64_PEAK_GINST = 2 * 152 * 2.07
# Warp-instructions per cell of the FP32 stage kernel (ncu smsp__inst_executed
# / cells, turbulent box 512^3, stage 1 / stage 2; profiles/) and the issue
# peak they run against: 4 warp-instructions per clock per SM (one per
# scheduler) x 152 SMs x 2.07 GHz.
FP32_WARP_INST_PER_CELL = {1: 74.19, 2: 80.10}
ISSUE_PEAK_GINST = 4 * 152 * 2.07
# FP64-pipe lane-instructions per cell of the FP64 WENO-Z stage kernel (ncu,
# Orszag-Tang 256^3; first / middle / last SSP-RK3 stage).
WENO_FP64_INST_PER_CELL = {"stage1": 3511.2, "stage_mid": 3529.2, "stage2": 3530.3}
# Warp-instructions per cell of the FP32 WENO-Z stage kernel (ncu
# smsp__inst_executed / cells, Orszag-Tang 256^3; first / middle / last
# SSP-RK3 stage).
WENO_FP32_WARP_INST_PER_CELL = {"stage1": 126.87, "stage_mid": 128.31, "stage2": 133.00}
# Algorithmic HBM bytes per cell: stage 1 reads U^n and writes U1 (18 words),
# stage 2 reads U1 and U^n and writes U^{n+1} (27 words).
WORDS_STAGE = {1: 18, 2: 27}
# SSP-RK3: the middle stage also reads U^n (27 words), like the last one.
WORDS_STAGE_RK3 = {"stage1": 18, "stage_mid": 27, "stage2": 27}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="edge of the FP64 OT grid")
    ap.add_argument("--n32", type=int, default=512, help="edge of the FP32 turbulent grid")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-brio", action="store_true", help="skip the Brio-Wu latency line")
    ap.add_argument("--no-paper-scheme", action="store_true",
                    help="skip the WENO-Z + SSP-RK3 throughput lines")
    ap.add_argument("--no-decomposed", action="store_true",
                    help="skip the line of the grid decomposed into blocks on one GPU")
    ap.add_argument("--mode", default="replicas", choices=["replicas", "decomposed"],
                    help="under torchrun: independent replicas (default), or one n^3 block per "
                         "rank of a grid decomposed along z, halos exchanged over NCCL")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(self.idx), "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


# -------------------------------------------------------------- CPU oracle --
def _cpu_problem(n: int):
    import oracle as orc
    from paper_2510_24175_gb300 import inputs
    pb = inputs.orszag_tang_3d(n)
    g = orc.Grid(n=pb.n, dx=pb.dx, gamma=pb.gamma, glm_alpha=pb.glm_alpha, limiter=pb.limiter,
                 bc=pb.bc, cfl=pb.cfl)
    return pb, g, orc.prim_to_cons(pb.prim(), pb.gamma)


def cpu_oracle_sample(n: int = 256, slab: int = 32):
    """Times the CPU FP64 oracle as it stands on the bench workload itself
    (3-D Orszag-Tang n^3, one RK2 step with its CFL wave-speed reduction):
    on all host cores through the slab-parallel runner (one process per
    core, each stepping a z slab with its ghost planes exchanged through
    shared memory; bitwise the single-process oracle), and on one core for a
    z slab of `slab` planes of the same grid (the same per-zone arithmetic)."""
    import oracle as orc
    from oracle.slab import SlabRunner
    pb, g, U0 = _cpu_problem(n)
    ncores = os.cpu_count() or 1
    with SlabRunner(g, nproc=ncores) as r:
        t0 = time.perf_counter()
        r.run(U0, 1)
        el = time.perf_counter() - t0
        nproc = r.nproc
    allc = pb.ncell / el
    # one core: one step of an n x n x slab periodic box with the same cells
    sub = orc.Grid(n=(n, n, slab), dx=g.dx, gamma=g.gamma, glm_alpha=g.glm_alpha,
                   limiter=g.limiter, bc=g.bc, cfl=g.cfl)
    Us = np.ascontiguousarray(U0[:, :slab])
    t0 = time.perf_counter()
    orc.run(Us, sub, 1)
    t1 = time.perf_counter() - t0
    single = n * n * slab / t1
    return {"value": allc, "unit": "zone-updates/s", "cores": nproc, "kind": "oracle",
            "sample": f"one RK2 step (with its CFL wave-speed reduction) of the 3-D "
                      f"Orszag-Tang {n}^3 workload itself on {nproc} host cores: {nproc} "
                      f"single-threaded oracle processes, one z slab each, ghost planes "
                      f"exchanged through shared memory ({el:.1f} s); single_thread_value: "
                      f"one RK2 step of an {n} x {n} x {slab} periodic box of the same cells "
                      f"(its first {slab} planes) in one process ({t1:.1f} s)",
            "single_thread_value": single, "host_cores": ncores}


def workload_config(n: int, world: int, t_reached=None) -> dict:
    cfg = {"workload": f"orszag_tang_3d_{n}^3_fp64", "n": [n, n, n],
           "limiter": "MC", "riemann": "HLLD+GLM", "time": "RK2", "cfl": 0.8,
           "l2": "state arrays (1.2 GB each at 256^3) larger than L2; no flush",
           "parallelism": f"{world} independent replica(s)"}
    if t_reached is not None:
        cfg["t_reached"] = t_reached
    return cfg


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on the bench workload
    itself (3-D Orszag-Tang n^3 FP64, MC, HLLD + GLM, RK2), every bench step
    one full step on all host cores through the slab-parallel runner."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle.slab import SlabRunner
    n = args.n
    pb, g, U0 = _cpu_problem(n)
    ncores = os.cpu_count() or 1
    with SlabRunner(g, nproc=ncores) as r:
        r.run(U0, max(args.warmup, 0))
        U = r.A.copy()
        t0 = time.perf_counter()
        res = r.run(U, args.steps)
        el = time.perf_counter() - t0
        nproc = r.nproc
    val = pb.ncell * args.steps / el
    sample = (f"each bench step: one full RK2 step (with its CFL wave-speed reduction) of the "
              f"{n}^3 Orszag-Tang workload on {nproc} host cores ({nproc} single-threaded "
              f"oracle processes, one z slab each, ghost planes exchanged through shared "
              f"memory; bitwise the single-process oracle); t reached {res.t:.6e}")
    print(json.dumps({
        "impl": "reference", "metric": "zone-updates/s", "value": val,
        "unit": "zone-updates/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (closed-form Orszag-Tang initial condition)",
        "config": {**workload_config(n, 1), "parallelism": f"{nproc} host processes (z slabs)"},
        "cpu_baseline": {"value": val, "unit": "zone-updates/s", "cores": nproc,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "zone-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


# ------------------------------------------------------------------- GPU --
def timed_steps(s, torch, K, dist, world):
    stream = torch.cuda.current_stream()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    s.profile(True)
    s.profile_read()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        s.step()
    e1.record(stream)
    torch.cuda.synchronize()
    prof = s.profile_read()
    s.profile(False)
    ms = e0.elapsed_time(e1)
    if dist is not None:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    return ms, prof


def fp64_peak_keys(ach, fma):
    """The measured FP64 peak beside the nominal one: mhd_fp64_fma_rate run
    on this GPU in this process (an FMA is one lane-instruction)."""
    if not fma:
        return {}
    pk = fma["lane_fma_per_s"] / 1e9
    return {"peak_measured": pk, "frac_of_measured": ach / pk,
            "peak_measured_source": "mhd_fp64_fma_rate on this GPU in this run: one CTA of 8 "
                                    "warps per SM, 16 independent DFMA chains per thread "
                                    f"({fma['lanes_per_clk_per_sm']:.2f} lanes/clk/SM)"}


def roofline_of(prof, ncell, esize, hbm_peak, peak_kind, fp64, fma=None):
    """Roofline of the stage kernel (both RK stages) from its CUDA-event times."""
    n1, ms1 = prof["stage1"]
    n2, ms2 = prof["stage2"]
    avg_ms = (ms1 + ms2) / max(n1 + n2, 1)
    bytes_launch = ncell * esize * (WORDS_STAGE[1] + WORDS_STAGE[2]) / 2.0
    tb = TRAFFIC_BYTES_PER_CELL.get(esize) if TRAFFIC_BYTES_PER_CELL else None
    traffic = ncell * (tb[1] * n1 + tb[2] * n2) / max(n1 + n2, 1) if tb else None
    hbm = {"bound": "hbm", "achieved": bytes_launch / (avg_ms * 1e-3) / 1e9, "peak": hbm_peak,
           "unit": "GB/s", "traffic": traffic, "kernel": "rk_stage_kernel",
           "avg_launch_ms": avg_ms, "bytes_per_launch": bytes_launch,
           "peak_source": peak_kind}
    hbm["frac"] = hbm["achieved"] / hbm_peak
    if not fp64:
        return hbm, None
    inst = ncell * (FP64_INST_PER_CELL[1] * n1 + FP64_INST_PER_CELL[2] * n2) / max(n1 + n2, 1)
    ach = inst / (avg_ms * 1e-3) / 1e9
    alu = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_GINST,
           "unit": "G FP64-lane-inst/s", "frac": ach / FP64_PEAK_GINST, "traffic": traffic,
           "kernel": "rk_stage_kernel", "avg_launch_ms": avg_ms,
           "fp64_inst_per_cell": FP64_INST_PER_CELL,
           "peak_source": "nominal: 2 FP64 lanes/clk/SM x 152 SMs x 2.07 GHz (GB300 "
                          "1.25 TFLOP/s FP64); the SM's FP64 unit is the bound",
           **fp64_peak_keys(ach, fma)}
    return hbm, alu


def run_decomposed(args):
    """--mode decomposed: one n^3 block per rank of an Orszag-Tang grid of
    n x n x (n ranks) cells on [0,1] x [0,1] x [0,ranks] (the vortex repeats
    along z, so every block does the single-box work), decomposed along z;
    per stage each rank packs its two z boundary slabs and exchanges them with
    its neighbours over NCCL, per step the wave speed is max-allreduced.
    Weak scaling; value = zone-updates/s of the whole grid."""
    import torch
    import torch.distributed as dist
    import paper_2510_24175_gb300 as m
    from paper_2510_24175_gb300 import inputs
    from paper_2510_24175_gb300.decomp import DistributedBlock
    from dataclasses import replace
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n, K, W = args.n, args.steps, args.warmup
    pb = inputs.orszag_tang_3d(n)
    cfg = replace(m.Config.from_problem(pb), n=(n, n, n * world), xmax=(1.0, 1.0, float(world)))
    blk = DistributedBlock(cfg, (1, 1, world), rank)
    mine = replace(pb, xmin=(0.0, 0.0, float(rank)), xmax=(1.0, 1.0, float(rank + 1)))
    blk.solver.set_state(torch.from_numpy(mine.prim()).cuda(), kind=m.MHD_PRIM)
    for _ in range(W):
        blk.step()
    stream = torch.cuda.current_stream()
    dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        blk.step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t = torch.tensor([e0.elapsed_time(e1)], device="cuda", dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    dist.barrier()
    if rank == 0:
        value = world * pb.ncell * K / (ms * 1e-3)
        print(json.dumps({
            "metric": "zone-updates/s", "value": value, "unit": "zone-updates/s",
            "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": ms / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (closed-form Orszag-Tang initial condition)",
            "config": {**workload_config(n, world),
                       "parallelism": f"grid of {n} x {n} x {n * world} cells decomposed along "
                                      f"z into {world} blocks, halo exchange over NCCL"},
            "clocks": clk}))
    dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.mode == "decomposed":
        run_decomposed(args)
        return
    import numpy as np
    import torch
    import paper_2510_24175_gb300 as m
    from paper_2510_24175_gb300 import inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    K, W = args.steps, args.warmup
    hbm_peak, peak_kind = peaks()
    fma = m.mhd_fp64_fma_rate()  # the FP64 rooflines' measured denominator

    # ---- FP64: 3-D Orszag-Tang 256^3 ------------------------------------
    pb = inputs.orszag_tang_3d(args.n)
    N = pb.ncell
    s = m.MHD(m.Config.from_problem(pb))
    V0 = torch.from_numpy(pb.prim()).cuda()
    s.set_state(V0, kind=m.MHD_PRIM)
    for _ in range(W):
        s.step()
    s.step_info()
    clocks = ClockSampler(local)
    clocks.start()
    ms, prof = timed_steps(s, torch, K, dist, world)
    clk = clocks.stop()
    info = s.step_info()
    value = world * N * K / (ms * 1e-3)
    hbm, alu = roofline_of(prof, N, 8, hbm_peak, peak_kind, True, fma)
    launches = sum(c for c, _ in prof.values())
    kernels = {k: {"launches": c, "total_ms": t, "avg_ms": (t / c if c else 0.0)}
               for k, (c, t) in prof.items()}

    # ---- end to end through the C ABI with pinned host buffers -------------
    e2e = None
    if not args.no_e2e:
        U_host = torch.empty((9,) + tuple(V0.shape[1:]), dtype=torch.float64, pin_memory=True)
        s.get_state(U_host.numpy())
        out_host = torch.empty(U_host.shape, dtype=torch.float64, pin_memory=True)
        Kx = max(3, min(K, 10))
        for _ in range(W):  # warm-up of the end-to-end loop itself
            s.step_host(U_host.numpy(), out_host.numpy())
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(Kx):
            s.step_host(U_host.numpy(), out_host.numpy())
        el = time.perf_counter() - t0
        if dist is not None:
            t = torch.tensor([el], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": world * N * Kx / el, "unit": "zone-updates/s",
               "h2d_bytes_per_step": int(U_host.numel() * 8),
               "d2h_bytes_per_step": int(out_host.numel() * 8), "steps": Kx,
               "api": "mhd_step_host (pinned host input and output every step; input "
                      "slabs overlap the wave-speed reduction, output halves overlap the "
                      "last stage)"}
    del s, V0
    torch.cuda.empty_cache()

    # ---- FP32 bulk: turbulent box 512^3 ----------------------------------
    fp32 = None
    if not args.no_fp32:
        pb32 = inputs.turbulent_box(args.n32)
        N32 = pb32.ncell
        s32 = m.MHD(m.Config.from_problem(pb32))
        V32 = torch.from_numpy(pb32.prim()).cuda()
        s32.set_state(V32, kind=m.MHD_PRIM)
        del V32
        for _ in range(W):
            s32.step()
        s32.step_info()
        ms32, prof32 = timed_steps(s32, torch, K, dist, world)
        s32.step_info()
        hbm32, _ = roofline_of(prof32, N32, 4, hbm_peak, peak_kind, False)
        n1, t1 = prof32["stage1"]
        n2, t2 = prof32["stage2"]
        winst = N32 * (FP32_WARP_INST_PER_CELL[1] * n1 + FP32_WARP_INST_PER_CELL[2] * n2)
        ach32 = winst / ((t1 + t2) * 1e-3) / 1e9
        issue32 = {"bound": "alu", "achieved": ach32, "peak": ISSUE_PEAK_GINST,
                   "unit": "G warp-inst/s", "frac": ach32 / ISSUE_PEAK_GINST,
                   "kernel": "rk_stage_kernel",
                   "peak_source": "4 warp-instructions/clk/SM (instruction issue) x 152 SMs x "
                                  "2.07 GHz; the FP32 kernel is issue-bound (ncu)"}
        fp32 = {"workload": f"turbulent_box_{args.n32}^3_fp32", "value": world * N32 * K / (ms32 * 1e-3),
                "unit": "zone-updates/s", "ms_per_step": ms32 / K, "roofline": hbm32,
                "roofline_issue": issue32,
                "kernels": {k: {"launches": c, "total_ms": t} for k, (c, t) in prof32.items()},
                "dtype": "f32 (FP64 dt reduction, sums, pressure-floor branch)"}
        launches += sum(c for c, _ in prof32.values())
        del s32
        torch.cuda.empty_cache()

    # ---- FP32 on the FP64 grid (same-grid precision ratio) -----------------
    fp32_same = None
    if not args.no_fp32:
        pbs = inputs.orszag_tang_3d(args.n)
        ss = m.MHD(m.Config.from_problem(pbs, precision=m.MHD_FP32))
        ss.set_state(torch.from_numpy(pbs.prim()).cuda(), kind=m.MHD_PRIM)
        for _ in range(W):
            ss.step()
        ss.step_info()
        mss, profs = timed_steps(ss, torch, K, dist, world)
        ss.step_info()
        fp32_same = {"workload": f"orszag_tang_3d_{args.n}^3_fp32",
                     "value": world * pbs.ncell * K / (mss * 1e-3), "unit": "zone-updates/s",
                     "ms_per_step": mss / K}
        launches += sum(c for c, _ in profs.values())
        del ss
        torch.cuda.empty_cache()

    # ---- FP64 on the FP32 sweep's grid (turbulent box 512^3) ---------------
    fp64_512 = None
    if not args.no_fp32:
        pbt = inputs.turbulent_box(args.n32)
        st = m.MHD(m.Config.from_problem(pbt, precision=m.MHD_FP64))
        Vt = torch.from_numpy(pbt.prim()).cuda()
        st.set_state(Vt, kind=m.MHD_PRIM)
        del Vt
        for _ in range(W):
            st.step()
        st.step_info()
        Kt = max(3, min(K, 5))
        mst, proft = timed_steps(st, torch, Kt, dist, world)
        st.step_info()
        fp64_512 = {"workload": f"turbulent_box_{args.n32}^3_fp64",
                    "value": world * pbt.ncell * Kt / (mst * 1e-3), "unit": "zone-updates/s",
                    "steps": Kt, "ms_per_step": mst / Kt}
        launches += sum(c for c, _ in proft.values())
        del st
        torch.cuda.empty_cache()

    # ---- Brio-Wu 1024 to t = 0.1 (latency-bound 1-D case): GPU wall time ----
    brio = None
    if not args.no_brio:
        pbb = inputs.brio_wu(1024)
        sb = m.MHD(m.Config.from_problem(pbb))
        Vb = pbb.prim()
        sb.set_state(torch.from_numpy(Vb).cuda(), kind=m.MHD_PRIM)
        nb = 0
        while sb.step_info()["t"] < pbb.t_end and nb < 100000:  # untimed: count the steps
            sb.step()
            nb += 1
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times = {}
        for mode in ("single", "graph", "graph"):  # the second graph run is timed
            sb.set_state(torch.from_numpy(Vb).cuda(), kind=m.MHD_PRIM)
            torch.cuda.synchronize()
            e0.record(stream)
            if mode == "single":
                for _ in range(nb):
                    sb.step()
            else:
                sb.step_n(nb)
            e1.record(stream)
            torch.cuda.synchronize()
            times[mode] = e0.elapsed_time(e1)
        brio = {"workload": "brio_wu_1024_fp64_to_t_0.1", "steps": nb,
                "t_reached": sb.step_info()["t"], "gpu_ms": times["graph"],
                "gpu_ms_single_launches": times["single"],
                "api": "mhd_step_n (the steps replayed from one captured CUDA graph)",
                "note": "state set from the device; the oracle's time for the same run is in "
                        "cpu_baseline"}
        del sb
        torch.cuda.empty_cache()

    # ---- the paper's own schemes, OT 256^3: WENO-Z + SSP-RK3 with GLM ------
    # ---- (its strong-scaling runs) or constrained transport (weak scaling) --
    paper_scheme = None
    if not args.no_paper_scheme:
        paper_scheme = {}
        Kp = max(3, min(K, 5))
        for divb, dtag in ((m.MHD_DIVB_GLM, "glm"), (m.MHD_DIVB_CT, "ct")):
            for prec, tag in ((m.MHD_FP64, "fp64"), (m.MHD_FP32, "fp32")):
                pw = inputs.orszag_tang_3d(args.n)
                pw.limiter, pw.rk_order, pw.divb = m.MHD_LIM_WENOZ, 3, divb
                sw = m.MHD(m.Config.from_problem(pw, precision=prec))
                sw.set_state(torch.from_numpy(pw.prim()).cuda(), kind=m.MHD_PRIM)
                if divb == m.MHD_DIVB_CT:
                    sw.set_face_field(torch.from_numpy(pw.faces()).cuda())
                for _ in range(W):
                    sw.step()
                sw.step_info()
                msw, profw = timed_steps(sw, torch, Kp, dist, world)
                sw.step_info()
                key = tag if divb == m.MHD_DIVB_GLM else f"ct_{tag}"
                paper_scheme[key] = {
                    "workload": f"orszag_tang_3d_{args.n}^3_wenoz_rk3_{dtag}_{tag}",
                    "value": world * pw.ncell * Kp / (msw * 1e-3), "unit": "zone-updates/s",
                    "steps": Kp, "ms_per_step": msw / Kp,
                    "kernels": {k: {"launches": c, "total_ms": t}
                                for k, (c, t) in profw.items() if c}}
                if divb == m.MHD_DIVB_CT:
                    paper_scheme[key]["divb_max_after"] = sw.divb_max()
                if prec == m.MHD_FP64 and divb == m.MHD_DIVB_GLM:
                    inst = sum(pw.ncell * WENO_FP64_INST_PER_CELL[c] * profw[c][0]
                               for c in WENO_FP64_INST_PER_CELL)
                    ms_k = sum(profw[c][1] for c in WENO_FP64_INST_PER_CELL)
                    ach = inst / (ms_k * 1e-3) / 1e9
                    paper_scheme[key]["roofline"] = {
                        "bound": "alu", "achieved": ach, "peak": FP64_PEAK_GINST,
                        "unit": "G FP64-lane-inst/s", "frac": ach / FP64_PEAK_GINST,
                        "kernel": "rk_stage_weno_kernel", **fp64_peak_keys(ach, fma)}
                if prec == m.MHD_FP32 and divb == m.MHD_DIVB_GLM:
                    # issue roofline (warp-instructions) and HBM fraction of
                    # the FP32 WENO-Z stage kernel
                    ms_k = sum(profw[c][1] for c in WORDS_STAGE_RK3)
                    if WENO_FP32_WARP_INST_PER_CELL:
                        winst = sum(pw.ncell * WENO_FP32_WARP_INST_PER_CELL[c] * profw[c][0]
                                    for c in WENO_FP32_WARP_INST_PER_CELL)
                        ach = winst / (ms_k * 1e-3) / 1e9
                        paper_scheme[key]["roofline_issue"] = {
                            "bound": "alu", "achieved": ach, "peak": ISSUE_PEAK_GINST,
                            "unit": "G warp-inst/s", "frac": ach / ISSUE_PEAK_GINST,
                            "kernel": "rk_stage_weno_kernel",
                            "warp_inst_per_cell": WENO_FP32_WARP_INST_PER_CELL}
                    nbytes = pw.ncell * 4 * sum(WORDS_STAGE_RK3[c] * profw[c][0]
                                                for c in WORDS_STAGE_RK3)
                    achb = nbytes / (ms_k * 1e-3) / 1e9
                    paper_scheme[key]["roofline"] = {
                        "bound": "hbm", "achieved": achb, "peak": hbm_peak, "unit": "GB/s",
                        "frac": achb / hbm_peak, "kernel": "rk_stage_weno_kernel",
                        "peak_source": peak_kind}
                launches += sum(c for c, _ in profw.values())
                if divb == m.MHD_DIVB_CT:  # edge, face and cell kernels per stage record
                    launches += 2 * profw["ct"][0]
                del sw
                torch.cuda.empty_cache()

    # ---- adjoint / forward step-time ratio: 2-D Orszag-Tang 512^2 FP64 ------
    adjoint = None
    if not args.no_adjoint:
        from paper_2510_24175_gb300.adjoint import rollout_solver
        pba = inputs.orszag_tang_2d(512)
        sa = rollout_solver(pba)
        sa.set_state(torch.from_numpy(pba.prim()).cuda(), kind=m.MHD_PRIM)
        for _ in range(W):
            sa.step()
        info_a = sa.step_info()
        dt_a, ch_a = info_a["dt"], info_a["ch"]
        Ka = max(K, 10)
        stream = torch.cuda.current_stream()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(Ka):
            sa.step(dt_a, ch_a)
        ev[1].record(stream)
        Ua = sa.get_state()
        U1a = torch.empty_like(Ua)
        # the reverse pass's forward recompute when it keeps the first stage
        ev[4].record(stream)
        for _ in range(Ka):
            sa.step(dt_a, ch_a)
            sa.get_stage1(U1a)
        ev[5].record(stream)
        lam = torch.randn_like(Ua)
        out = torch.empty_like(Ua)
        for _ in range(W):
            sa.adjoint_step(Ua, lam, out, dt_a, ch_a)
            sa.adjoint_step_stage1(Ua, U1a, lam, out, dt_a, ch_a)
        torch.cuda.synchronize()
        ev[2].record(stream)
        for i in range(Ka):
            if i % 2 == 0:
                sa.adjoint_step(Ua, lam, out, dt_a, ch_a)
            else:
                sa.adjoint_step(Ua, out, lam, dt_a, ch_a)
        ev[3].record(stream)
        ev[6].record(stream)
        for i in range(Ka):
            if i % 2 == 0:
                sa.adjoint_step_stage1(Ua, U1a, lam, out, dt_a, ch_a)
            else:
                sa.adjoint_step_stage1(Ua, U1a, out, lam, dt_a, ch_a)
        ev[7].record(stream)
        torch.cuda.synchronize()
        ms_f = ev[0].elapsed_time(ev[1]) / Ka
        ms_a = ev[2].elapsed_time(ev[3]) / Ka
        ms_fk = ev[4].elapsed_time(ev[5]) / Ka
        ms_ak = ev[6].elapsed_time(ev[7]) / Ka
        adjoint = {"workload": "orszag_tang_2d_512^2_fp64", "forward_ms_per_step": ms_f,
                   "adjoint_ms_per_step": ms_a,
                   "adjoint_over_forward": ms_ak / ms_f,
                   "adjoint_over_forward_checkpointed": (ms_ak + ms_fk) / ms_f,
                   "forward_keep_stage1_ms_per_step": ms_fk,
                   "adjoint_stage1_kept_ms_per_step": ms_ak,
                   "adjoint_over_forward_recomputing_stage1": (ms_a + ms_f) / ms_f,
                   "note": "adjoint_over_forward = one adjoint step using the step's kept "
                           "state and first RK stage (adjoint_step_stage1) / one forward "
                           "step: the backward pass of MHDRollout with k = 0, which keeps "
                           "both in HBM during the forward pass (two 18.9 MB states per "
                           "step); _checkpointed adds the step's forward recompute that "
                           "keeps its first stage (MHDRollout with k > 0, all but a "
                           "segment's last step)"}
        # forward FP64 step: prep, two stages, exact speed pass; 2-D adjoint:
        # init, stage-1 recompute, 2 x (primitives, 2 face sweeps, cells)
        launches += 2 * Ka * 4 + Ka * 10 + Ka * 9
        del sa
        torch.cuda.empty_cache()

    # ---- batched ensemble: 64 seeded boxes, FP32, 10 steps, one launch -----
    ensemble = None
    if not args.no_ensemble:
        sizes, b0s = inputs.ensemble_sizes(64, seed=5)
        pbs = []
        for n_, b0 in zip(sizes, b0s):
            pbe = inputs.orszag_tang_3d(n_)
            pbe.params = {"B0": b0}
            pbe.precision = m.MHD_FP32
            pbs.append(pbe)
        cfgs = [m.Config.from_problem(q) for q in pbs]
        ens = m.Ensemble(cfgs)
        for b, q in enumerate(pbs):
            ens.set_state(b, torch.from_numpy(q.prim()).cuda(), kind=m.MHD_PRIM)
        Ke = 10
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def time_ens():
            ens.step(Ke)  # warm-up; builds the graph for Ke-step launches
            torch.cuda.synchronize()
            e0.record(stream)
            ens.step(Ke)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)

        ms_fixed = time_ens()  # the fixed 32 x 8 tiles, z chunks of 16
        for b, q in enumerate(pbs):
            ens.set_state(b, torch.from_numpy(q.prim()).cuda(), kind=m.MHD_PRIM)
        ens.autotune(2)
        ms_e = time_ens()
        shapes = {}
        for b, q in enumerate(pbs):
            inf = ens.info(b)
            shapes[f"{q.n[0]}^3"] = f"32x{inf['ty']} tiles, {inf['tz']}-plane z chunks"
        cells = sum(q.ncell for q in pbs)
        plain = [m.MHD(c) for c in cfgs]
        for b, q in enumerate(pbs):
            plain[b].set_state(torch.from_numpy(q.prim()).cuda(), kind=m.MHD_PRIM)
            plain[b].step()
        torch.cuda.synchronize()
        e0.record(stream)
        for s_ in plain:
            for _ in range(Ke):
                s_.step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_p = e0.elapsed_time(e1)
        ensemble = {"workload": "64 boxes, edges from {32,48,64,96,128} (seed 5), OT with "
                                "B0 in [0.1,0.5], FP32, 10 steps",
                    "cells": cells, "graph": ens.info(0)["graph"],
                    "persistent_value": cells * Ke / (ms_e * 1e-3),
                    "per_box_plain_value": cells * Ke / (ms_p * 1e-3),
                    "unit": "zone-updates/s", "speedup_vs_plain": ms_p / ms_e,
                    "autotuned_shapes": shapes,
                    "fixed_32x8_value": cells * Ke / (ms_fixed * 1e-3),
                    "speedup_autotuned_vs_fixed_32x8": ms_fixed / ms_e}
        launches += 1 + Ke * 3 * len(plain)
        del ens, plain
        torch.cuda.empty_cache()

    # ---- the same grid as 2 x 2 blocks on this GPU (halo faces) ------------
    decomposed = None
    if not args.no_decomposed:
        from paper_2510_24175_gb300.decomp import LocalBlocks
        dims = (1, 2, 2)
        lb = LocalBlocks(m.Config.from_problem(pb), dims)
        lb.set_state(torch.from_numpy(pb.prim()).cuda(), kind=m.MHD_PRIM)
        for _ in range(W):
            lb.step()
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        for b in lb.blocks:
            b.profile(True)
            b.profile_read()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            lb.step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_d = e0.elapsed_time(e1)
        reads = [b.profile_read() for b in lb.blocks]  # a read clears the record
        stage_ms = sum(r[c][1] for r in reads for c in ("stage1", "stage2"))
        halo_bytes = sum(b.halo_bytes(f) for r, b in enumerate(lb.blocks)
                         for f in lb.dec.halo_faces(r))
        decomposed = {
            "workload": f"orszag_tang_3d_{args.n}^3_fp64 as {dims[1]} x {dims[2]} blocks (y, z) "
                        "on one GPU, halo buffers packed from the neighbouring blocks each stage",
            "value": N * K / (ms_d * 1e-3), "unit": "zone-updates/s", "ms_per_step": ms_d / K,
            "stage_kernels_ms_per_step": stage_ms / K,
            "over_undecomposed": (N * K / (ms_d * 1e-3)) / value,
            "halo_bytes_per_stage": int(halo_bytes)}
        del lb
        torch.cuda.empty_cache()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    cpu = None
    if not args.no_cpu and world == 1:
        cpu = cpu_oracle_sample()
        if brio is not None:  # the oracle on the same Brio-Wu run, one process
            import oracle as orc
            pbb = inputs.brio_wu(1024)
            g = orc.Grid(n=pbb.n, dx=pbb.dx, gamma=pbb.gamma, glm_alpha=pbb.glm_alpha,
                         limiter=pbb.limiter, bc=pbb.bc, cfl=pbb.cfl)
            U0 = orc.prim_to_cons(pbb.prim(), pbb.gamma)
            t0 = time.perf_counter()
            r = orc.run(U0, g, 100000, t_end=pbb.t_end)
            cpu["brio_wu_1024_oracle_s"] = time.perf_counter() - t0
            cpu["brio_wu_1024_oracle_t"] = r.t

    line = {
        "metric": "zone-updates/s", "value": value, "unit": "zone-updates/s",
        "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": ms / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (closed-form Orszag-Tang initial condition)",
        "config": workload_config(args.n, world, info["t"]),
        "roofline": alu if alu is not None else hbm,
        "roofline_hbm": hbm,
        "kernels": kernels,
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": e2e,
        "fp32": fp32,
        "fp32_same_grid": fp32_same,
        "fp32_over_fp64_same_grid": (fp32_same["value"] / value) if fp32_same else None,
        "fp64_turbulent_512": fp64_512,
        "fp32_over_fp64_turbulent_512": (fp32["value"] / fp64_512["value"])
        if (fp32 and fp64_512) else None,
        "brio_wu": brio,
        "paper_scheme_wenoz_rk3": paper_scheme,
        "adjoint": adjoint,
        "ensemble": ensemble,
        "decomposed_one_gpu": decomposed,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
