"""Benchmark of the FP64 RHS + SSP-RK3 stage on one B300 (per rank).

Default workload: the 3D inert shock-bubble interaction with 5 species
(512 x 256 x 256, viscous + diffusion, Ma drawn by seed 0), the paper's
roofline headline case. One "step" is one full SSP-RK3 step (three stages of
the whole hot path) over the synthetic field. The metric is FP64 cell-updates
per RK3 stage per second (cells x 3 x steps / time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (oracle/, plain FP64 C++) on a bounded
sample of the same workload on the host cores. Prints ONE JSON line on rank 0.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64 cell-updates/s per RK3 stage (1 B300), % HBM roofline; batched & adjoint vs plain"
UNIT = "cell-stage updates/s"
WORKLOADS = {
    # name: (config index, grid)
    "sbi3d_n5": (2, None),
    "sbi2d_n3": (1, None),
}
FP64_NOMINAL_TFLOPS = 1.25   # B300 dense FP64 (nominal), reported beside the measured probe
# ncu figures of k_face on the 3D 5-species case (160x80x80, one launch per
# direction; profiles/k_face_sbi3d_n5_160x80x80.md): DRAM bytes (mean of the
# three directions) and executed FP64 flops (DFMA = 2) per face, valid only for the
# kernel source they were taken on (first 16 hex digits of the sha256 of
# xf_device.cuh); any other source reports them as null.
FACE_NCU = {"source": "366890e7a68936f3", "dram_bytes_per_face": 366.7,
            "fp64_flops_executed_per_face": 1804.0}
# bounded oracle samples of each workload (config index -> grid)
CPU_SAMPLE_GRID = {2: (96, 48, 48), 1: (256, 128)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6400.0, "source": "fallback"}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out, _ = self.p.communicate()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if "Active" in f[3 + k] and "Not" not in f[3 + k]:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max(value, device=None):
    """Maximum of a float over all ranks (the value itself when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, seconds_max, world):
    """Units processed by all ranks (each rank does the same replica) per second
    of the slowest rank."""
    return world * units_per_rank / seconds_max


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _cpu_baseline(cfg=2, steps=5, warmup=1):
    """Time the oracle on a bounded sample of the workload on the host cores:
    ``warmup`` untimed steps, then ``steps`` steps timed one by one; the rate
    is that of the median step (the spread of the steps beside it)."""
    from paper_2403_05910_b300 import cases
    from oracle.xfo import Oracle
    cores = len(os.sched_getaffinity(0))
    grid = CPU_SAMPLE_GRID[cfg]
    case = cases.config(cfg, n=grid)
    o = Oracle(case, threads=cores)
    U, T = o.prim_to_cons()
    dt = o.dt(U, T)
    for _ in range(max(1, warmup)):
        o.step(U, T, dt)
    times = []
    for _ in range(max(3, steps)):
        t0 = time.perf_counter()
        o.step(U, T, dt)
        times.append(time.perf_counter() - t0)
    med = statistics.median(times)
    rate = [case.cells * 3 / t for t in times]
    return {"value": case.cells * 3 / med, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(times)} RK3 steps timed one by one (median), after "
                      f"{max(1, warmup)} untimed, of the same setup ({case.name}) on a "
                      f"{'x'.join(map(str, grid))} grid ({case.cells} cells)",
            "grid": list(grid), "seconds": sum(times), "median_step_s": med,
            "spread": [min(rate), max(rate)]}


def _cpu_baseline_as_reference_arm(args):
    """The cpu_baseline leg, measured by running this script's reference arm
    (``--impl reference``) in a process of its own, so that both legs time the
    oracle in the same kind of process: one without torch or CUDA, whose
    OpenMP runtime state differs from this one's."""
    env = {k: v for k, v in os.environ.items()
           if k not in ("RANK", "LOCAL_RANK", "WORLD_SIZE", "MASTER_ADDR", "MASTER_PORT")}
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--impl", "reference",
                          "--steps", "5", "--warmup", "3", "--workload", args.workload],
                         capture_output=True, text=True, env=env, check=True).stdout
    line = json.loads(out.strip().splitlines()[-1])
    cb = dict(line["cpu_baseline"])
    cb["sample"] += "; run as this script's reference arm in a process of its own"
    return cb


def _cpu_single_core(cfg=2, steps=3):
    """The oracle on one host core (the kind of CPU figure GPU speed-ups are
    usually quoted against), on a smaller sample of the same workload."""
    from paper_2403_05910_b300 import cases
    from oracle.xfo import Oracle
    grid = {2: (48, 24, 24), 1: (128, 64)}[cfg]
    case = cases.config(cfg, n=grid)
    o = Oracle(case, threads=1)
    U, T = o.prim_to_cons()
    dt = o.dt(U, T)
    o.step(U, T, dt)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        o.step(U, T, dt)
        times.append(time.perf_counter() - t0)
    med = statistics.median(times)
    return {"value": case.cells * 3 / med, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} RK3 steps timed one by one (median) on a "
                      f"{'x'.join(map(str, grid))} grid ({case.cells} cells)",
            "seconds": sum(times)}


def _config(case, ws):
    """The workload description both arms print."""
    return {"workload": f"{case.name}: {'x'.join(str(n) for n in case.n[:case.dim])}, "
                        f"{case.n_species} species, viscous+diffusion, "
                        f"Ma={case.params['Ma']:.4f}, r={case.params['r']}H",
            "cells": case.cells, "n_v": case.n_v,
            "l2": "working set > 126 MB L2 (state + per-cell fields ~"
                  f"{(case.n_v * 2 + 34) * case.cells * 8 / 1e9:.0f} GB): no flush needed",
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"}


def _workload_meta(args):
    """Name, grid, species and draws of the workload without building its
    fields (the draws do not depend on the grid)."""
    import dataclasses
    from paper_2403_05910_b300 import cases
    cfg, grid = WORKLOADS[args.workload]
    small = cases.config(cfg, n=(8, 4, 4) if cfg == 2 else (8, 4))
    full = grid or {2: (512, 256, 256), 1: (1024, 512)}[cfg]
    if args.grid:
        full = tuple(int(x) for x in args.grid.split(","))
    n = tuple(list(full) + [1] * (3 - len(full)))
    return dataclasses.replace(small, n=n, prim=None)


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import build as ob
    ob.build()
    cfg = WORKLOADS[args.workload][0]
    cb = _cpu_baseline(cfg, steps=args.steps, warmup=args.warmup)
    config = _config(_workload_meta(args), ws)
    grid = "x".join(map(str, cb["grid"]))
    config["workload"] += (f"; the oracle is timed on a {grid} sample of the same setup "
                           f"(the rate per cell-stage does not depend on the grid size)")
    config["timed_grid"] = grid
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * cb["median_step_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _batched_vs_per_instance(args, dev, stream):
    """The 64-instance 2D shock-bubble ensemble: one persistent kernel per stage
    (autotuned, CUDA graph) against per-instance xf_step_rk3 launches on the
    same stream; aggregate cell-stage updates/s of each."""
    import torch
    from paper_2403_05910_b300 import cases
    from paper_2403_05910_b300.xf import Batch, Solver
    cs = cases.batch(0)
    cells = sum(c.cells for c in cs)
    b = Batch(cs)
    for i, c in enumerate(cs):
        b.set_primitive(i, torch.from_numpy(c.prim).to(dev))
    choice, ms_cand = b.autotune(steps=1, report=True)
    shape = b.config()

    def timed(fn, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    for _ in range(args.warmup):
        b.step(0.0)
    ms_b = timed(lambda: b.step(0.0), args.steps)
    st_b = b.status()
    graph = b.uses_graph()
    b.close()
    ss = [Solver(c) for c in cs]
    for sv, c in zip(ss, cs):
        sv.set_primitive(torch.from_numpy(c.prim).to(dev))

    def per():
        for sv in ss:
            sv.step(0.0)

    for _ in range(args.warmup):
        per()
    ms_p = timed(per, args.steps)
    for sv in ss:
        sv.close()
    return {"workload": "64 2D viscous shock-bubble instances, 128x64..768x384, N 3-5, seed 0",
            "instances": len(cs), "cells": cells, "unit": UNIT,
            "value": cells * 3 / (ms_b * 1e-3), "per_instance_value": cells * 3 / (ms_p * 1e-3),
            "speedup": ms_p / ms_b, "ms_per_step": ms_b, "per_instance_ms_per_step": ms_p,
            "autotuned_shape": {"block_threads": shape[0], "tile_w": shape[1], "tile_h": shape[2]},
            "candidates_ms_per_step": [round(x, 2) for x in ms_cand],
            "cuda_graph": graph, "status_flags": st_b}


def _rounds_ms(fns, k, stream, reset=None, rounds=5):
    """Per-call time (ms) of each function: in each of `rounds` rounds every
    function in turn runs k times back to back between two CUDA events on the
    launch stream (after `reset`, untimed, when given), so a clock change moves
    all of them alike; the median round of each. One untimed call each first."""
    import torch
    for fn in fns:
        if reset:
            reset()
        fn()
    ts = [[] for _ in fns]
    for _ in range(rounds):
        for i, fn in enumerate(fns):
            if reset:
                reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(k):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts[i].append(e0.elapsed_time(e1) / k)
    return [sorted(t)[len(t) // 2] for t in ts]


def _adjoint_vs_forward(args, dev, stream):
    """The differentiated workload (2D shock-bubble, 512x256, 4 species): time
    of one RHS adjoint against one forward RHS, of one RK3-step adjoint
    (from taped stage states, and recomputing them) against one step, and of
    the whole checkpointed gradient against its forward pass."""
    import torch
    from paper_2403_05910_b300 import cases
    from paper_2403_05910_b300.xf import Solver
    c = cases.config(4)
    s = Solver(c)
    s.set_primitive(torch.from_numpy(c.prim).to(dev))
    for _ in range(args.warmup):
        s.step(0.0)
    dtd = torch.zeros(1, dtype=torch.float64, device=dev)
    s.compute_dt(dtd)
    dt = 0.9 * float(dtd.item())
    U = torch.empty((c.n_v, c.cells), dtype=torch.float64, device=dev)
    T0 = torch.empty(c.cells, dtype=torch.float64, device=dev)
    s.get_state(U, T0)
    R = torch.empty_like(U)
    W = torch.randn(U.shape, dtype=torch.float64, generator=torch.Generator().manual_seed(0)).to(dev)
    Ub = torch.zeros_like(U)

    k = max(args.steps, 5)
    reset = lambda: s.set_state(U, T0)   # the state and its warm start
    f, a = _rounds_ms([lambda: s.rhs(U, R), lambda: s.rhs_adjoint(U, W, Ub)], k, stream)
    U1, U2 = torch.empty_like(U), torch.empty_like(U)
    reset()
    s.step_tape(dt, U1, U2)
    fs, at, ar = _rounds_ms([lambda: s.step(dt), lambda: s.step_adjoint_tape(dt, U1, U2, Ub),
                             lambda: s.step_adjoint(dt, Ub)], k, stream, reset)
    st = s.status()
    grad = _gradient_timing(s, c, dt, dev, stream)
    st |= s.status()
    s.close()
    options = {name: _adjoint_option(c, kw, dt, W, k, dev, stream) for name, kw in ADJ_OPTIONS}
    return {"workload": "sbi2d_n4_adjoint: 512x256, 4 species, viscous, fixed dt",
            "rhs_ms": f, "rhs_adjoint_ms": a, "rhs_ratio": a / f,
            "step_ms": fs, "step_adjoint_ms": at, "step_ratio": at / fs,
            "step_adjoint_recompute_ms": ar, "step_ratio_recompute": ar / fs,
            "note": "step adjoint from the taped stage states (xf_step_rk3_adjoint_tape); "
                    "the recompute form rebuilds the two intermediate stage states itself",
            "options": options, "gradient": grad, "status_flags": st}


ADJ_OPTIONS = (("weno_cu6", {"weno": 6}), ("weno7", {"weno": 7}),
               ("mixture_averaged_diffusion", {"diffusion": 1}),
               ("weno5+positivity", {"positivity": True}))


def _adjoint_option(c, kw, dt, W, k, dev, stream):
    """One option of the path on the differentiated workload: RHS and RHS
    adjoint, step and step adjoint (taped; with the blend, from the stage
    states and the flux tape; and recomputing), in ms."""
    import torch
    from paper_2403_05910_b300 import cases
    from paper_2403_05910_b300.xf import Solver
    case = cases.with_binary_diffusion(c) if kw.get("diffusion") else c
    s = Solver(case, **kw)
    s.set_primitive(torch.from_numpy(c.prim).to(dev))
    U = torch.empty((c.n_v, c.cells), dtype=torch.float64, device=dev)
    T0 = torch.empty(c.cells, dtype=torch.float64, device=dev)
    s.get_state(U, T0)
    R, Ub = torch.empty_like(U), torch.zeros_like(U)

    f, a = _rounds_ms([lambda: s.rhs(U, R), lambda: s.rhs_adjoint(U, W, Ub)], k, stream)
    U1, U2 = torch.empty_like(U), torch.empty_like(U)
    Fh = (torch.empty(s.tape_flux_len(), dtype=torch.float64, device=dev)
          if kw.get("positivity") else None)
    s.set_state(U, T0)
    s.step_tape(dt, U1, U2, Fhat=Fh)
    fs, at, ar = _rounds_ms([lambda: s.step(dt),
                             lambda: s.step_adjoint_tape(dt, U1, U2, Ub, Fhat=Fh),
                             lambda: s.step_adjoint(dt, Ub)], k, stream,
                            lambda: s.set_state(U, T0))
    st = s.status()
    s.close()
    return {"rhs_ms": f, "rhs_adjoint_ms": a, "rhs_ratio": a / f, "step_ms": fs,
            "step_adjoint_taped_ms": at, "step_ratio_taped": at / fs,
            "step_adjoint_recompute_ms": ar, "step_ratio_recompute": ar / fs,
            "flux_tape": Fh is not None, "status_flags": st}


def _gradient_timing(s, c, dt, dev, stream):
    """dJ/dP0 of the differentiated workload as specified: 200 fixed-dt RK3
    steps, a checkpoint every 20, J = sum Y_3 (1 - Y_3) dV, through
    torch.autograd (taped backward). Forward-only time beside it."""
    import torch
    from paper_2403_05910_b300.autodiff import mixing_after_steps
    steps, every = 200, 20

    def run(n, grad):
        P0 = torch.from_numpy(c.prim).to(dev).requires_grad_(grad)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        J = mixing_after_steps(P0, s, dt, n, every, 2)
        if grad:
            J.backward()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    run(every, True)   # warm-up: allocations, first calls
    fwd = run(steps, False)
    both = run(steps, True)
    return {"steps": steps, "checkpoint_every": every, "forward_ms": fwd,
            "forward_backward_ms": both, "ratio": both / fwd}


VARIANTS = (("weno5+positivity", {"positivity": True}), ("weno_cu6", {"weno": 6}),
            ("weno7", {"weno": 7}), ("mixture_averaged_diffusion", {"diffusion": 1}))


def _variants(args, dev, stream, case):
    """The same workload and step with the other options of the path: WENO5
    with the positivity-preserving blend (Eq. 17-20), WENO-CU6, WENO7, and
    the mixture-averaged diffusion of Eq. 25-26 (seeded binary fits added to
    the same species). Rate and the face kernels' FP64 rate from the
    library's own events."""
    import torch
    from paper_2403_05910_b300 import cases, flops
    from paper_2403_05910_b300.xf import Solver
    steps = max(1, min(args.steps, 5))
    out = {}
    case_dsm = cases.with_binary_diffusion(case)
    for name, kw in VARIANTS:
        s = Solver(case_dsm if kw.get("diffusion") else case, **kw)
        P = torch.from_numpy(case.prim).to(dev)
        s.set_primitive(P)
        del P
        for _ in range(args.warmup):
            s.step(0.0)
        s.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            s.step(0.0)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = s.profile_read()
        ms = e0.elapsed_time(e1)
        st = s.status()
        s.close()
        fl = flops.per_cell_stage(case, weno=kw.get("weno", 5), positivity=kw.get("positivity", False),
                                  diffusion=kw.get("diffusion", 0))
        face_ms = sum(prof[k][0] for k in ("face_x", "face_y", "face_z") if k in prof)
        face_n = sum(prof[k][1] for k in ("face_x", "face_y", "face_z") if k in prof)
        face_tf = fl["face"] / case.dim / (face_ms / face_n * 1e-3) / 1e12
        out[name] = {"value": case.cells * 3 * steps / (ms * 1e-3), "unit": UNIT,
                     "ms_per_step": ms / steps, "steps": steps,
                     "face_fp64_tflops": face_tf, "face_frac_of_nominal": face_tf / FP64_NOMINAL_TFLOPS,
                     "flops_per_face": flops.face(case.dim, case.n_species, case.viscous,
                                                  kw.get("weno", 5), kw.get("positivity", False),
                                                  kw.get("diffusion", 0)),
                     "kernels_ms_per_step": {k: v[0] / steps for k, v in prof.items()},
                     "status_flags": st}
    return out


def run_ours(args):
    import numpy as np
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2403_05910_b300 import build, cases, flops
    build.build()
    from paper_2403_05910_b300.xf import Solver, probe_fp64

    cfg, grid = WORKLOADS[args.workload]
    if args.grid:
        grid = tuple(int(x) for x in args.grid.split(","))
    case = cases.config(cfg, n=grid)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    s = Solver(case)
    P = torch.from_numpy(case.prim).to(dev)
    s.set_primitive(P)
    del P
    for _ in range(args.warmup):
        s.step(0.0)
    torch.cuda.synchronize()
    assert s.status() == 0, "non-physical state during warm-up"

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region (per-kernel events on the same stream)
    s.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            s.step(0.0)
        ev1.record(stream)
        barrier()
    prof = s.profile_read()
    s.profile(False)
    ms = ev0.elapsed_time(ev1)
    ms_all = reduce_max(ms, dev)
    status = s.status()
    cell_stages = case.cells * 3 * args.steps
    value = whole_job_rate(cell_stages, ms_all * 1e-3, ws)
    # kernels launched: one per profiled region, plus the ghost-layer copy
    # (k_ghost) that follows k_prim in each primitive-recovery region
    launches = sum(n for _, n in prof.values())
    launches += prof.get("prim", (0.0, 0))[1]

    # ---- roofline of the dominant kernel class (the face-flux kernels)
    fl = flops.per_cell_stage(case)
    face_ms = sum(prof[k][0] for k in ("face_x", "face_y", "face_z") if k in prof)
    face_n = sum(prof[k][1] for k in ("face_x", "face_y", "face_z") if k in prof)
    face_flops_per_launch = fl["face"] / case.dim
    achieved = face_flops_per_launch / (face_ms / face_n * 1e-3) / 1e12
    fp64_probe = probe_fp64()
    import hashlib
    with open(os.path.join(ROOT, "paper_2403_05910_b300", "csrc", "xf_device.cuh"), "rb") as f:
        src_hash = hashlib.sha256(f.read()).hexdigest()[:16]
    faces_per_launch = fl["face"] / case.dim / flops.face(case.dim, case.n_species, case.viscous)
    ncu_ok = FACE_NCU["source"] == src_hash
    bpf = FACE_NCU["dram_bytes_per_face"] if ncu_ok else None
    xpf = FACE_NCU["fp64_flops_executed_per_face"] if ncu_ok else None
    traffic = None if bpf is None else bpf * faces_per_launch
    executed = None if xpf is None else xpf * faces_per_launch / (face_ms / face_n * 1e-3) / 1e12
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", 6400.0)
    alg_bytes = sum(flops.hbm_bytes_per_cell_stage(case, st) for st in range(3)) / 3.0
    hbm_achieved = alg_bytes * cell_stages / (ms * 1e-3) / 1e9

    # ---- end to end through the C-ABI with host buffers: every step uploads
    # U^n and T from pinned host memory and reads U^{n+1} and T back
    # (xf_step_rk3_host: the copies overlap the compute in slabs)
    Uh = torch.empty((case.n_v, case.cells), dtype=torch.float64).pin_memory()
    Th = torch.empty(case.cells, dtype=torch.float64).pin_memory()
    s.get_state(Uh, Th)
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.step_host(Uh, Th, Uh, Th, 0.0)
        torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - t0, dev)
    e2e_val = whole_job_rate(case.cells * 3 * e2e_steps, e2e_s, ws)
    io_bytes = (case.n_v + 1) * case.cells * 8
    s.close()
    variants = None if args.no_variants else _variants(args, dev, stream, case)
    batched = None if args.no_batch else _batched_vs_per_instance(args, dev, stream)
    adjoint = None if args.no_adjoint else _adjoint_vs_forward(args, dev, stream)

    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            from oracle import build as ob
            ob.build()
            cpu = _cpu_baseline_as_reference_arm(args)
            cpu["single_core"] = _cpu_single_core(cfg)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(case, ws),
            "roofline": {"bound": "alu", "kernel": "k_face (x, y, z face fluxes)",
                         "achieved": achieved, "peak": fp64_probe, "unit": "TFLOP/s",
                         "frac": achieved / fp64_probe,
                         "peak_note": "the library's FP64 FMA probe (independent DFMA "
                                      "chains on every SM) measured in this run; achieved "
                                      "counts the method's flops per face (flops.py: "
                                      "per-cell eigenvalues of the LLF maxima count "
                                      "per cell, not per face)",
                         "peak_nominal": FP64_NOMINAL_TFLOPS,
                         "frac_of_nominal": achieved / FP64_NOMINAL_TFLOPS,
                         "executed": executed,
                         "frac_executed": None if executed is None else executed / fp64_probe,
                         "executed_note": "ncu-counted FP64 flops per face of this source "
                                          "(DFMA = 2) per launch duration; null when the "
                                          "counters were taken on another source",
                         "flops_per_face": flops.face(case.dim, case.n_species, case.viscous),
                         "traffic": traffic, "traffic_unit": "B per launch",
                         "kernel_source": src_hash},
            "hbm_roofline": {"achieved": hbm_achieved, "peak": hbm, "unit": "GB/s",
                             "frac": hbm_achieved / hbm,
                             "alg_bytes_per_cell_stage": alg_bytes},
            "stage_flops_per_cell": fl["total"] / case.cells,
            "fp64_tflops_whole_step": fl["total"] * 3 * args.steps / (ms * 1e-3) / 1e12,
            "kernels_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
            "gpu_launches": launches,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": io_bytes,
                    "d2h_bytes_per_step": io_bytes, "steps": e2e_steps},
            "clocks": clk.summary(),
            "status_flags": status,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if variants is not None:
            line["variants"] = variants
        if batched is not None:
            line["batched"] = batched
        if adjoint is not None:
            line["adjoint"] = adjoint
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="sbi3d_n5")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-vs-per-instance leg")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint-vs-forward leg")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the positivity / WENO-CU6 / WENO7 / mixture-diffusion leg")
    ap.add_argument("--grid", default="", help="override the grid, e.g. 160,80,80 (profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)  # at least three untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
