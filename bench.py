#!/usr/bin/env python
"""Benchmark: unknowns/s to a 1e-10 relative residual on the 3D AMR Poisson
workload (octree of 8^3 blocks, base 128^3 plus 3 refinement levels in
nested spheres around a seeded Gaussian source, ~20M unknowns, Dirichlet
values from the closed-form potential).

One step = one full solve from phi = 0 to a composite relative residual of
1e-10: FP32 cycles inside FP64 defect correction (the headline), and the
plain FP64 FMG + V-cycle solve measured the same way.  Inputs are resident
in HBM when the timed region starts; the working set (~1.5 GB) is far larger
than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The line also carries "batch": the 512-tree cylindrical forest solved as one
batch (mixed precision and FP64, per-tree relative residual 1e-10), and
"mesh": the construction of a uniform 1024^3 grid of 16^3 blocks (the case
Sec. 2.5 quotes 0.3 s for) and one adaptation of it.

N > 1 (torchrun): every rank solves its own replica (the workload is one
tree; the method does not shard here), value = all ranks' unknowns / max
time.  --impl reference times the FP64 CPU oracle on a bounded sample.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "unknowns/s to 1e-10 rel. residual (FP64 vs FP32+defect corr.); V-cycle HBM GB/s vs peak"
WORKLOAD = ("3D Cartesian Poisson eps=1, octree of 8^3 blocks, base 128^3 + 3 refinement levels in nested "
            "spheres (r = 0.30/0.22/0.14) around a Gaussian source (sigma = 0.02, centre seeded in [0.3,0.7]^3), "
            "Dirichlet from the closed-form potential")
TOL = 1e-10
MAX_CYCLES = 40


def problem():
    from synth import workloads as W
    return W.cfg2_gauss3d(base=128, N=8, seed=0)


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in d:
                v = d[k]
                return float(v["value"] if isinstance(v, dict) else v), "measured"
    except Exception:
        pass
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_sha1(name):
    """sha1 of one kernel template's source text in mg_kernels.cu."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_1901_11370_gb300", "csrc", "mg_kernels.cu")).read()
    i = src.index(name + "(")
    start = src.rfind("template", 0, i)
    end = src.index("\n}\n", i) + 3
    return hashlib.sha1(src[start:end].encode()).hexdigest()


def measured_traffic(kernel, fname):
    """DRAM bytes per cell from a committed ncu summary (entries of
    "key: value" lines separated by blank lines), or None when the kernel
    has no entry or its source changed since the capture."""
    path = os.path.join(ROOT, "profiles", fname)
    try:
        text = "".join(ln for ln in open(path) if not ln.startswith("#"))
        for entry in text.split("\n\n"):
            kv = dict(ln.split(":", 1) for ln in entry.splitlines() if ":" in ln)
            kv = {k.strip(): v.strip() for k, v in kv.items()}
            if kv.get("kernel") == kernel and kv.get("source_sha1") == kernel_sha1(kernel):
                return float(kv["dram_bytes_per_cell"])
    except Exception:
        pass
    return None


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def oracle_solve_time(o, threads):
    """Wall seconds of one full FP64 oracle solve from phi = 0 to a composite
    relative residual of 1e-10 (FMG, then V-cycles, the schedule the GPU
    runs), with `threads` threads over the blocks of each level."""
    import oracle
    used = oracle.set_threads(threads)
    t0 = time.perf_counter()
    cycles, hist = o.solve(TOL, MAX_CYCLES)
    dt = time.perf_counter() - t0
    return dt, cycles, hist[-1] / hist[0], used


def oracle_baseline(p, n_leaf):
    """The FP64 C oracle timed on this host: the full solve of the benchmark
    workload to 1e-10, once on every host core (OpenMP over the blocks of a
    level; the result is bit-identical for any thread count) and once on a
    single core.  Mesh construction and input setup are not timed."""
    from oracle import Oracle
    o = Oracle.from_problem(p)
    cores = os.cpu_count() or 1
    dt_all, cyc, rel, used = oracle_solve_time(o, cores)
    dt_one, cyc1, _, _ = oracle_solve_time(o, 1)
    import oracle
    oracle.set_threads(cores)
    return {"value": n_leaf / dt_all, "unit": "unknowns/s", "cores": used, "kind": "oracle",
            "host_cpus": cores, "cycles_to_tol": cyc, "final_rel_residual": rel, "seconds": dt_all,
            "sample": "one full solve (FMG + %d V-cycles to 1e-10) of the FP64 C oracle on the full %d-unknown "
                      "workload, %d threads" % (cyc - 1, n_leaf, used),
            "single_thread": {"value": n_leaf / dt_one, "cores": 1, "seconds": dt_one, "cycles_to_tol": cyc1}}


def run_reference(args):
    """The reference arm: the FP64 C oracle (the paper's method written out
    plainly), one full solve to 1e-10 of the benchmark workload per step on
    every host core.  Rank 0 alone under torchrun."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from oracle import Oracle
    from synth import workloads as W
    p = problem()
    n_leaf = W.n_leaf_cells(p)
    o = Oracle.from_problem(p)
    cores = os.cpu_count() or 1
    times, cyc, rel, used = [], 0, 0.0, 1
    for s in range(args.warmup + args.steps):
        dt, cyc, rel, used = oracle_solve_time(o, cores)
        if s >= args.warmup:
            times.append(dt)
    per = sum(times) / len(times)
    value = n_leaf / per
    sample = ("each step: one full solve (FMG + %d V-cycles, phi = 0 to 1e-10 relative residual) of the FP64 C "
              "oracle on the full %d-unknown workload, %d threads" % (cyc - 1, n_leaf, used))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "unknowns": n_leaf, "cycles_to_tol": cyc,
                                          "final_rel_residual": rel, "parallelism": "%d host threads" % used},
           "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": used, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def solve_alg_bytes(levels, n_leaf, cycles, precision, dim=3, down=None, up=None, inner=1):
    """Algorithmic HBM bytes of one solve by the per-cell minimum traffic of
    its cycles (each sweep reads x and f once and writes x once; the
    transfers read and write each level once; constant coefficient), for
    the schedule the solve ran (down[l] + up[l] sweeps on level l, -1 or
    None meaning 2; `inner` V-cycles per outer step): per level cell and
    cycle, FP32 cycles 12 B per sweep + 20 B (3D; 24 in 2D) for the
    residual, restriction, prolongation and coarse terms, FP64 cycles 24 B
    per sweep + 40 B (48 in 2D) -- 68 and 136 B at V(2,2) in 3D.  Per outer
    step and leaf, FP32 cycles in FP64 defect correction add the FP64
    residual (read phi and f, write the FP32 defect: 20 B) and the update
    (read e, phi, write phi: 20 B); FP64 solves the composite residual (read
    phi, f: 16 B).  The coarsest level is solved directly (no sweeps).  FMG
    counts as one outer step."""
    def steps(a, l):
        return 2 if a is None or l >= len(a) or a[l] < 0 else int(a[l])
    per_cycle, level_cells = 0, 0
    for l, L in enumerate(levels):
        cells = L["nb"] * L["n"] ** dim
        level_cells += cells
        sw = 0 if l == 0 else steps(down, l) + steps(up, l)
        if precision == "fp64":
            per_cycle += cells * (24 * sw + (40 if dim == 3 else 48))
        else:
            per_cycle += cells * (12 * sw + (20 if dim == 3 else 24))
    per = inner * per_cycle + (16 if precision == "fp64" else 40) * n_leaf
    return cycles * per, level_cells


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    from paper_1901_11370_gb300 import build as B
    if rank == 0:
        B.build()
    if dist is not None:
        dist.barrier()
    import paper_1901_11370_gb300 as mg
    from synth import workloads as W

    p = problem()
    tree = mg.Tree.from_problem(p)
    n = tree.n_leaf
    zeros = torch.zeros(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    # sweeps per level and inner cycles per outer step: the schedule
    # autotuner (mg_tune_schedule), once per precision, untimed like the
    # sweep-kernel autotuner; each precision is timed with its own choice
    sched = {}
    for prec in (mg.MG_FP32_DC, mg.MG_FP64):
        tree.set_schedule()
        inner, _ = tree.tune_schedule(TOL, MAX_CYCLES, prec)
        d, u = tree.schedule()
        sched[prec] = (d.copy(), u.copy(), inner)

    def solve(prec):
        d, u, inner = sched[prec]
        tree.set_schedule(d, u)
        tree.set_phi(zeros)
        return tree.solve(TOL, MAX_CYCLES, fmg_first=True, precision=prec, inner_cycles=inner)

    def timed(prec, steps):
        barrier()
        l0 = tree.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = None
        for _ in range(steps):
            info = solve(prec)
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1) / steps
        return max_over_ranks(ms), info, tree.launch_count() - l0

    for _ in range(args.warmup):
        solve(mg.MG_FP32_DC)
        solve(mg.MG_FP64)

    clocks = Clocks(local)
    clocks.start()
    ms_mixed, (cyc_mixed, rel_mixed), launches = timed(mg.MG_FP32_DC, args.steps)
    ms64, (cyc64, rel64), launches64 = timed(mg.MG_FP64, args.steps)
    clk = clocks.stop()

    # end to end through the public API: every step uploads its rhs from
    # pinned host memory, runs set_rhs / set_phi / solve / get_phi, and reads
    # its phi back into pinned host memory.  The copies run on their own
    # stream with two buffers each, so step k's read-back and step k+1's
    # upload overlap the neighbouring solves; every step still moves its own
    # bytes inside the timed region, which ends when the last read-back has.
    rhs_host = torch.from_numpy(W.leaf_field(p, "rhs")).pin_memory()
    out_host = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(2)]
    rhs_dev = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(2)]
    phi_dev = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(2)]
    copy = torch.cuda.Stream()
    up = [torch.cuda.Event() for _ in range(2)]    # rhs_dev[s] holds the step's rhs
    used = [torch.cuda.Event() for _ in range(2)]  # set_rhs has read rhs_dev[s]
    done = [torch.cuda.Event() for _ in range(2)]  # phi_dev[s] holds the step's phi
    down = [torch.cuda.Event() for _ in range(2)]  # out_host[s] has been read back

    def upload(k):
        s = k % 2
        copy.wait_event(used[s])
        with torch.cuda.stream(copy):
            rhs_dev[s].copy_(rhs_host, non_blocking=True)
        up[s].record(copy)

    def e2e_step(k):
        s = k % 2
        stream.wait_event(up[s])
        tree.set_rhs(rhs_dev[s])
        used[s].record(stream)
        tree.set_phi(zeros)
        tree.solve(TOL, MAX_CYCLES, fmg_first=True, precision=mg.MG_FP32_DC, inner_cycles=sched[mg.MG_FP32_DC][2])
        stream.wait_event(down[s])
        tree.get_phi(out=phi_dev[s])
        done[s].record(stream)
        copy.wait_event(done[s])
        with torch.cuda.stream(copy):
            out_host[s].copy_(phi_dev[s], non_blocking=True)
        down[s].record(copy)

    def e2e_run(steps):
        upload(0)
        for k in range(steps):
            if k + 1 < steps:
                upload(k + 1)
            e2e_step(k)
        stream.wait_event(down[(steps - 1) % 2])

    tree.set_schedule(*sched[mg.MG_FP32_DC][:2])
    e2e_run(2)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    copy.wait_stream(stream)
    e2e_run(args.steps)
    e1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    assert torch.equal(out_host[(args.steps - 1) % 2], phi_dev[(args.steps - 1) % 2].cpu())

    # roofline of the dominant kernel (fused red-black sweep) on the largest
    # level.  Algorithmic bytes: 12 B per cell per FP32 sweep (read x and f
    # once, write x once), i.e. 6 B per cell for one colour launch, 12 B in
    # FP64; the DRAM bytes ncu measured for the same launch are reported
    # beside it
    (ms_s, ms_g, b_s, b_g), lev = tree.time_sweeps(n_sweeps=8, precision=mg.MG_FP32_DC)
    (ms_s64, _, b_s64, _), _ = tree.time_sweeps(n_sweeps=4, precision=mg.MG_FP64)
    peak, peak_kind = peak_hbm()
    lv = tree.levels()[lev]
    lev_cells = lv["nb"] * lv["n"] ** 3
    alg = 6.0 * lev_cells
    achieved = alg / (ms_s * 1e-3) / 1e9
    var32 = tree.sweep_variant(lev, mg.MG_FP32_DC)
    var64 = tree.sweep_variant(lev, mg.MG_FP64)
    kname = {0: "k_sweep_tma", 1: "k_sweep", 2: "k_sweep_warp", 3: "k_sweep_warp", 4: "k_sweep_rows",
             5: "k_sweep_rows", 6: "k_sweep_flat", 7: "k_sweep_rows", 8: "k_sweep_rows",
             9: "k_sweep_rows", 10: "k_sweep_tma"}.get(var32, "k_sweep")
    traffic = measured_traffic(kname, "sweep_f32_traffic.txt")
    if traffic is not None:
        traffic *= lev_cells
    levels = tree.levels()
    sb32, level_cells = solve_alg_bytes(levels, n, cyc_mixed, "fp32_dc", down=sched[mg.MG_FP32_DC][0],
                                        up=sched[mg.MG_FP32_DC][1], inner=sched[mg.MG_FP32_DC][2])
    sb64, _ = solve_alg_bytes(levels, n, cyc64, "fp64", down=sched[mg.MG_FP64][0], up=sched[mg.MG_FP64][1],
                              inner=sched[mg.MG_FP64][2])

    total_unknowns = n * world
    value = total_unknowns / (ms_mixed * 1e-3)
    result = {
        "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "unknowns": n, "global_batch": world, "precision":
                   "FP32 red-black GS cycles inside FP64 defect correction, FP64 coarsest solve",
                   "schedule": {name: {"down": [int(v) for v in sched[prec][0]], "up": [int(v) for v in sched[prec][1]],
                                       "inner_cycles": int(sched[prec][2])}
                                for name, prec in (("fp32_dc", mg.MG_FP32_DC), ("fp64", mg.MG_FP64))},
                   "schedule_from": "mg_tune_schedule (sweeps per level and inner cycles, timed solves to 1e-10; "
                                    "level 0 is solved directly)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2: working set ~%.1f GB (FP64 + FP32 fields) vs 129 MB L2, "
                         "no flush" % (n * 60 / 1e9),
                   "cycles_to_tol": cyc_mixed, "final_rel_residual": rel_mixed},
        "fp64": {"value": total_unknowns / (ms64 * 1e-3), "ms_per_step": ms64, "cycles_to_tol": cyc64,
                 "final_rel_residual": rel64, "gpu_launches_per_step": launches64 / args.steps},
        "clocks": clk,
        "e2e": {"value": total_unknowns / (e2e_ms * 1e-3), "unit": "unknowns/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8,
                "copies": "pinned host buffers, own stream, double-buffered (overlap the neighbouring solves)"},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": "%s, FP32, one colour, level %d (autotuned variant %d: %s)" % (
                         kname, lev, var32, tree.SWEEP_VARIANTS.get(var32)),
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "alg_bytes_per_launch": alg, "alg_bytes_per_cell": 6.0, "level_cells": lev_cells,
                     "ms_per_launch": ms_s,
                     "achieved_dram_GBs": None if traffic is None else traffic / (ms_s * 1e-3) / 1e9,
                     "achieved_dram_frac": None if traffic is None else traffic / (ms_s * 1e-3) / 1e9 / peak,
                     "fp64_sweep": {"ms_per_launch": ms_s64, "alg_bytes_per_cell": 12.0,
                                    "achieved_GBs": 12.0 * lev_cells / (ms_s64 * 1e-3) / 1e9,
                                    "variant": tree.SWEEP_VARIANTS.get(var64)},
                     "ghost_fill_ms_per_launch": ms_g, "ghost_fill_achieved_GBs": b_g / (ms_g * 1e-3) / 1e9,
                     "solve": {"alg_bytes_fp32_dc": sb32, "alg_bytes_fp64": sb64, "level_cells": level_cells,
                               "frac_fp32_dc": sb32 / (ms_mixed * 1e-3) / 1e9 / peak,
                               "frac_fp64": sb64 / (ms64 * 1e-3) / 1e9 / peak}},
    }
    if not args.no_batch:
        del tree
        result["batch"] = batch_measure(args, mg, W, barrier, max_over_ranks)
    if not args.no_cfg3:
        result["cfg3"] = cfg3_measure(args, mg, W, barrier, max_over_ranks)
    if args.cfg5_base > 0:
        result["cfg5"] = cfg5_measure(args, mg, W, barrier, max_over_ranks, args.cfg5_base)
    if not args.no_mesh and rank == 0:
        try:
            result["mesh"] = mesh_measure(mg)
        except Exception as e:  # the headline line stands without it
            result["mesh"] = {"error": str(e)[:200]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = oracle_baseline(p, n)
    if rank == 0:
        print(json.dumps(result))
    if dist is not None:
        dist.destroy_process_group()


CFG3_WORKLOAD = ("3D variable-coefficient Poisson, 256^3 uniform in 16^3 blocks, eps = 100 inside a seeded sphere "
                 "of radius 0.25 and 1 outside, Neumann on the x faces and periodic in y and z, right-hand side a "
                 "zero-mean Gaussian random field (correlation length 0.05)")


def cfg3_measure(args, mg, W, barrier, max_over_ranks):
    """The variable-coefficient workload at its stated size: FP32 cycles in
    FP64 defect correction and plain FP64, each from phi = 0 to 1e-10 (the
    zero-mean solution of this singular problem); the relative difference of
    the two solutions; and the adjoint of L = 1/2 sum V (phi - t)^2 (t an
    independent Gaussian random field, seed 1, scaled to rms(phi)) solved to
    a relative adjoint residual of 1e-10, dL/df and dL/deps both returned."""
    import torch
    world, _, _ = dist_env()
    p = W.cfg3_varcoef3d()
    t = mg.Tree.from_problem(p)
    n = t.n_leaf
    zeros = torch.zeros(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    steps = max(1, min(args.steps, 3))
    out = {"workload": CFG3_WORKLOAD, "unknowns": n * world}
    phis = {}
    for name, prec in (("fp32_dc", mg.MG_FP32_DC), ("fp64", mg.MG_FP64)):
        # the schedule autotuner (sweeps per level, inner cycles), untimed
        # like the headline's; then the default V(2,2) schedule is put back
        # for the adjoint below
        inner, _ = t.tune_schedule(TOL, 80, prec)
        down, up = t.schedule()
        t.set_phi(zeros)
        t.solve(TOL, 80, fmg_first=True, precision=prec, inner_cycles=inner)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            t.set_phi(zeros)
            cyc, rel = t.solve(TOL, 80, fmg_first=True, precision=prec, inner_cycles=inner)
        e1.record(stream)
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1) / steps)
        phis[name] = t.get_phi().clone()
        out[name] = {"value": n * world / (ms * 1e-3), "unit": "unknowns/s", "ms_per_step": ms, "cycles_to_tol": cyc,
                     "final_rel_residual": rel,
                     "schedule": {"down": [int(x) for x in down], "up": [int(x) for x in up], "inner_cycles": inner}}
        t.set_schedule(None)
    d = phis["fp32_dc"] - phis["fp64"]
    out["fp32_dc_vs_fp64_rel_err"] = float(d.norm() / phis["fp64"].norm())
    g1 = W.random_field(256, 0.05, 1, 3)
    I, J, K, _ = W.leaf_cell_index(p)
    tgt = torch.from_numpy(g1[I, J, K]).cuda()
    phi = phis["fp64"]
    tgt *= phi.pow(2).mean().sqrt() / tgt.pow(2).mean().sqrt()
    g = (phi - tgt) / n
    t.set_phi(phi)
    lams = {}
    for key, prec in (("adjoint", mg.MG_FP32_DC), ("adjoint_fp64", mg.MG_FP64)):
        t.adjoint(g, rel_tol=TOL, max_cycles=120, precision=prec)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lams[key] = t.adjoint(g, rel_tol=TOL, max_cycles=120, precision=prec)[0]
        e1.record(stream)
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1))
        it, rel = t.last_adjoint
        out[key] = {"ms": ms, "iterations": it, "final_rel_residual": rel,
                    "unknowns_per_s": n * world / (ms * 1e-3), "outputs": "dL/df and dL/deps (FP64)",
                    "precision": ("FP32 V(2,2) cycles in the FP64 defect correction of the adjoint"
                                  if prec == mg.MG_FP32_DC else "FP64 V(2,2) cycles")}
    out["adjoint"]["rel_diff_vs_fp64"] = float((lams["adjoint"] - lams["adjoint_fp64"]).norm()
                                               / lams["adjoint_fp64"].norm())
    del t
    torch.cuda.empty_cache()
    return out


CFG5_WORKLOAD = ("3D divergence cleaning on a periodic %d^3-base octree of 16^3 blocks, 2 levels refined where max |B| "
                 "of a block is in the top 10%%, B a k^-5/3 Gaussian field (rms 1) plus a non-solenoidal blob "
                 "(peak 3 rms, width 0.05); FP32 cycles in FP64 defect correction to 1e-10, then the adjoint of "
                 "L = 1/2 sum V |B_new - B_t|^2")


def cfg5_measure(args, mg, W, barrier, max_over_ranks, base):
    """The cleaning workload: inputs from the seeded generator (k^-5/3 field
    plus blob, refinement by the |B| decile; not timed), one cleaning step
    (div B, zero-mean projection, FP32 + FP64 defect-correction solve to
    1e-10, B - grad phi: mg_clean) and the adjoint pass for
    L = 1/2 sum V |B_new - B_t|^2 with B_t an independent k^-5/3 field
    (mg_clean_adjoint to an adjoint residual of 1e-10), each timed with CUDA
    events after one warm-up run."""
    import torch
    world, _, _ = dist_env()
    t0 = time.perf_counter()
    ci = W.CleanInputs(n=base, N=16)
    p = ci.problem
    B = torch.from_numpy(ci.leaf_fields()).cuda()
    Bt = torch.from_numpy(ci.target()).cuda()
    gen_s = time.perf_counter() - t0
    t = mg.Tree.from_problem(p)
    n = t.n_leaf
    vol = t.leaf_volumes()
    stream = torch.cuda.current_stream()
    out = {"workload": CFG5_WORKLOAD % base, "unknowns": n * world, "refinements": len(ci.refine),
           "input_generation_s": gen_s}

    def timed(fn):
        fn()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        barrier()
        return max_over_ranks(e0.elapsed_time(e1)), r

    ms, (Bn, f, cyc, rel) = timed(lambda: t.clean(B, TOL, 60, precision=mg.MG_FP32_DC))
    out["clean"] = {"ms": ms, "value": n * world / (ms * 1e-3), "unit": "unknowns/s", "cycles_to_tol": cyc,
                    "final_rel_residual": rel, "div_B_l2_before": float(f.norm()),
                    "precision": "FP32 V(2,2) cycles in FP64 defect correction"}
    gBn = vol * (Bn - Bt)
    ms, gB = timed(lambda: t.clean_adjoint(gBn, TOL, 80, precision=mg.MG_FP32_DC))
    it, rel = t.last_adjoint
    out["adjoint"] = {"ms": ms, "unknowns_per_s": n * world / (ms * 1e-3), "iterations": it,
                      "final_rel_residual": rel, "outputs": "dL/dB (3 FP64 components)",
                      "precision": "FP32 V(2,2) cycles in the FP64 defect correction of the adjoint"}
    ms64, gB64 = timed(lambda: t.clean_adjoint(gBn, TOL, 80))
    it64, rel64 = t.last_adjoint
    out["adjoint_fp64"] = {"ms": ms64, "unknowns_per_s": n * world / (ms64 * 1e-3), "iterations": it64,
                           "final_rel_residual": rel64,
                           "rel_diff_vs_fp32_dc": float((gB - gB64).norm() / gB64.norm())}
    del t, B, Bt, Bn, gBn, gB, gB64, f
    torch.cuda.empty_cache()
    return out


BATCH_WORKLOAD = ("batch of 512 independent 2D cylindrical (r,z) trees, side 16k cells with k ~ U{2..32} in 16^2 "
                  "blocks, 0-2 AMR levels around a seeded ring point, eps = 1 + 0.5 sin(2 pi z), Dirichlet 0 at "
                  "r = 1, z = 0, z = 1, axis at r = 0, Gaussian source of width 0.03")


def batch_measure(args, mg, W, barrier, max_over_ranks):
    """The batched form: every tree of the forest solved to 1e-10 (per-tree
    relative residual) in one pool, FP32 + FP64 defect correction against
    the plain FP64 cycles, each solve one graph-replayed sequence.  With
    N > 1 ranks the 512 trees are split by unknowns (no data exchanged while
    solving); the time is the slowest rank's, the unknowns all ranks'."""
    import numpy as np
    import torch
    from paper_1901_11370_gb300.shard import gather_tree_values, shard_by_cost
    world, rank, _ = dist_env()
    all_probs = [W.cyl_ring_tree(i) for i in range(512)]
    mine = list(range(512))
    if world > 1:
        mine = shard_by_cost([W.n_leaf_cells(q) for q in all_probs], world)[rank]
    probs = [all_probs[i] for i in mine]
    b = mg.Batch([mg.Tree.from_problem(q, finalize=False) for q in probs])
    b.set_eps(torch.from_numpy(np.concatenate([W.leaf_field(q, "eps") for q in probs])).cuda())
    b.set_rhs(torch.from_numpy(np.concatenate([W.leaf_field(q, "rhs") for q in probs])).cuda())
    zeros = torch.zeros(b.n_leaf, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    inner = {}

    def solve(prec):
        b.set_phi(zeros)
        return b.solve(TOL, MAX_CYCLES, fmg_first=True, precision=prec, inner_cycles=inner[prec])

    total = b.n_leaf
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([float(b.n_leaf)], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt)
        total = int(tt.item())
    out = {"workload": BATCH_WORKLOAD, "trees": 512, "unknowns": total, "segments": len(b.segments()),
           "coarse": b.coarse_info(),
           "parallelism": "single GPU" if world == 1 else
           "%d ranks, trees split by unknowns, no data exchange while solving" % world}
    steps = max(1, min(args.steps, 3))
    for name, prec in (("fp32_dc", mg.MG_FP32_DC), ("fp64", mg.MG_FP64)):
        # sweeps per segment and inner cycles: the batch schedule autotuner,
        # untimed, right before this precision is timed
        inner[prec], _ = b.tune_schedule(TOL, MAX_CYCLES, prec)
        solve(prec)
        barrier()
        l0 = b.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            cyc, rel = solve(prec)
        e1.record(stream)
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1) / steps)
        rels = list(rel)
        if world > 1:
            rels = gather_tree_values(rels, mine, 512)
            cyc = int(max_over_ranks(float(cyc)))
        out[name] = {"value": total / (ms * 1e-3), "unit": "unknowns/s", "ms_per_step": ms, "cycles_to_tol": cyc,
                     "inner_cycles": inner[prec],
                     "max_final_rel_residual": float(max(rels)), "gpu_launches_per_step": (b.launch_count() - l0) / steps}
    out["fp32_dc_over_fp64"] = out["fp32_dc"]["value"] / out["fp64"]["value"]
    (ms_s, _, b_s, _), seg = b.time_sweeps(n_sweeps=8, precision=mg.MG_FP32_DC)
    peak, peak_kind = peak_hbm()
    out["sweep_roofline"] = {"segment": seg, "blocks": b.segments()[seg]["nb"], "ms_per_launch": ms_s,
                             "alg_bytes_per_launch": b_s, "achieved": b_s / (ms_s * 1e-3) / 1e9, "peak": peak,
                             "peak_kind": peak_kind, "frac": b_s / (ms_s * 1e-3) / 1e9 / peak}
    return out


def mesh_measure(mg):
    """Mesh construction and adaptation (Sec. 2.5, "Adapting the grid
    structure"): a uniform 1024^3 grid of 16^3 blocks (262,144 leaf blocks),
    the size the paper quotes about 0.3 s for, then mg_tree_adapt refining
    the base blocks within 0.1 of the centre.  Times are wall seconds from
    mg_tree_build_times: mesh tables (built on the device), device setup
    (allocation, uploads, coarsest-level inverse), FP64 sweep autotuning,
    and for the adapted tree the phi transfer; host_build_tables_s is the
    host construction of the same tables, for comparison."""
    import numpy as np
    import torch
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    t = mg.Tree(3, 16, 0, (0,) * 6, (0.0,) * 6, (1024,) * 3, (0.0,) * 3, (1.0,) * 3)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    bt = t.build_times()
    nb = 1024 // 16
    c = (np.arange(nb) + 0.5) / nb - 0.5
    r = np.sqrt(c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2)
    add = [(0, i, j, k) for k, j, i in zip(*np.nonzero(r < 0.1))]
    w0 = time.perf_counter()
    t1 = t.adapt(add)
    torch.cuda.synchronize()
    wall1 = time.perf_counter() - w0
    bt1 = t1.build_times()
    th = mg.Tree(3, 16, 0, (0,) * 6, (0.0,) * 6, (1024,) * 3, (0.0,) * 3, (1.0,) * 3, finalize=False, build_on=1)
    out = {"workload": "uniform 1024^3 grid of 16^3 blocks, Dirichlet 0 (construction; the paper: about 0.3 s)",
           "leaf_blocks": nb ** 3, "tables_on": t.built_on(), "tables_s": bt[0], "device_setup_s": bt[1],
           "autotune_s": bt[2], "wall_s": wall, "host_build_tables_s": th.build_times()[0],
           "adapt": {"refined_blocks": len(add), "leaf_cells": t1.n_leaf, "tables_on": t1.built_on(),
                     "tables_s": bt1[0], "device_setup_s": bt1[1], "autotune_s": bt1[2],
                     "phi_transfer_s": bt1[3], "wall_s": wall1}}
    del t1, t, th
    torch.cuda.empty_cache()
    return out


def run_profile(kind, pins="", inner=1, up=-1):
    """Small fixed launch sequences for ncu captures (not a benchmark):
    sweeps64 -- one red-black sweep (2 smoother + 2 ghost launches) on the
    largest level of the workload; solve32 / solve64 -- one solve after one
    untimed warm-up solve.  pins ("level:variant,...") fixes the sweep kernel
    per level after autotuning: the tuner's timings mean nothing under a
    profiler, which slows every launch, so a capture pins what a plain run of
    the same command printed."""
    import torch
    import paper_1901_11370_gb300 as mg
    torch.cuda.set_device(0)
    tree = mg.Tree.from_problem(problem())
    zeros = torch.zeros(tree.n_leaf, dtype=torch.float64, device="cuda")
    if kind in ("sweeps64", "sweeps32"):
        prec = mg.MG_FP64 if kind == "sweeps64" else mg.MG_FP32_DC
        tree.time_sweeps(n_sweeps=1, precision=prec)  # first use: allocation and autotuning
        pin_sweeps(tree, prec, pins)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("measure")
        tree.time_sweeps(n_sweeps=1, precision=prec)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    else:
        prec = mg.MG_FP32_DC if kind == "solve32" else mg.MG_FP64
        tree.time_sweeps(n_sweeps=1, precision=prec)  # autotuning
        pin_sweeps(tree, prec, pins)
        for rep in range(2):  # the second solve (graphs captured, tuning done) in the NVTX range
            tree.set_phi(zeros)
            torch.cuda.synchronize()
            if rep:
                torch.cuda.nvtx.range_push("measure")
            tree.solve(TOL, MAX_CYCLES, fmg_first=True, precision=prec, inner_cycles=inner,
                       n_up=up if up > 0 else 2)
            torch.cuda.synchronize()
            if rep:
                torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    print("profile %s done: %d launches" % (kind, tree.launch_count()))


def run_profile_cfg3(kind, steps=2):
    """The 256^3 variable-coefficient workload (contrast 100) for ncu launch
    lists: `steps` outer steps of a solve from phi = 0 (FMG first) after one
    untimed warm-up of the same call, the second inside the NVTX range
    "measure"; cfg3_32 runs FP32 cycles in FP64 defect correction, cfg3_64
    plain FP64."""
    import torch
    import paper_1901_11370_gb300 as mg
    from synth import workloads as W
    torch.cuda.set_device(0)
    tree = mg.Tree.from_problem(W.cfg3_varcoef3d())
    prec = mg.MG_FP32_DC if kind == "cfg3_32" else mg.MG_FP64
    zeros = torch.zeros(tree.n_leaf, dtype=torch.float64, device="cuda")
    for rep in range(2):
        tree.set_phi(zeros)
        torch.cuda.synchronize()
        if rep:
            torch.cuda.nvtx.range_push("measure")
        tree.solve(TOL, steps, fmg_first=True, precision=prec, raise_on_fail=False)  # stops after `steps`
        torch.cuda.synchronize()
        if rep:
            torch.cuda.nvtx.range_pop()
    print("sweep variants by level:", ",".join("%d:%d" % (l, tree.sweep_variant(l, prec))
                                              for l in range(len(tree.levels()))))
    print("profile %s done: %d launches" % (kind, tree.launch_count()))


def pin_sweeps(tree, prec, pins):
    for item in filter(None, pins.split(",")):
        lev, var = (int(x) for x in item.split(":"))
        tree.set_sweep_variant(var, level=lev, precision=prec)
    print("sweep variants by level:", ",".join("%d:%d" % (l, tree.sweep_variant(l, prec))
                                              for l in range(len(tree.levels()))))


def run_profile_batch(ntrees=512, inner=1):
    """One mixed-precision solve of the batch (the first `ntrees` trees of
    the 512-tree forest) after a warm-up solve, the second inside the NVTX
    range "measure" (for ncu launch lists and single-kernel captures)."""
    import numpy as np
    import torch
    import paper_1901_11370_gb300 as mg
    from synth import workloads as W
    torch.cuda.set_device(0)
    probs = [W.cyl_ring_tree(i) for i in range(ntrees)]
    b = mg.Batch([mg.Tree.from_problem(q, finalize=False) for q in probs])
    b.set_eps(torch.from_numpy(np.concatenate([W.leaf_field(q, "eps") for q in probs])).cuda())
    b.set_rhs(torch.from_numpy(np.concatenate([W.leaf_field(q, "rhs") for q in probs])).cuda())
    zeros = torch.zeros(b.n_leaf, dtype=torch.float64, device="cuda")
    for rep in range(2):
        b.set_phi(zeros)
        torch.cuda.synchronize()
        if rep:
            torch.cuda.nvtx.range_push("measure")
        b.solve(TOL, MAX_CYCLES, fmg_first=True, precision=mg.MG_FP32_DC, inner_cycles=inner)
        torch.cuda.synchronize()
        if rep:
            torch.cuda.nvtx.range_pop()
    print("segments (n, group, blocks, covered, coarsest):",
          " ".join("%d/%d/%d/%d/%d" % (q["n"], q["group"], q["nb"], q["nref"], q["coarsest"]) for q in b.segments()))
    print("profile batch32 done: %d launches" % b.launch_count())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-tree batch measurement")
    ap.add_argument("--no-mesh", action="store_true", help="skip the 1024^3 mesh construction measurement")
    ap.add_argument("--no-cfg3", action="store_true", help="skip the 256^3 variable-coefficient workload")
    ap.add_argument("--cfg5-base", type=int, default=512,
                    help="base grid of the divergence-cleaning workload (0: skip it)")
    ap.add_argument("--profile", choices=["sweeps64", "sweeps32", "solve32", "solve64", "batch32", "cfg3_32", "cfg3_64"],
                    default=None)
    ap.add_argument("--trees", type=int, default=512, help="with --profile batch32: trees of the forest to use")
    ap.add_argument("--inner", type=int, default=1,
                    help="with --profile solve* / batch32: FP32 cycles per outer step (the tuned schedule's choice)")
    ap.add_argument("--n-up", type=int, default=-1,
                    help="with --profile solve*: post-smoothing sweeps (the tuned schedule's choice; default 2)")
    ap.add_argument("--pin-sweeps", default="",
                    help="with --profile sweeps*/solve*: 'level:variant,...' sweep kernels to pin after tuning")
    args = ap.parse_args()
    if args.profile == "batch32":
        run_profile_batch(args.trees, args.inner)
    elif args.profile in ("cfg3_32", "cfg3_64"):
        run_profile_cfg3(args.profile)
    elif args.profile:
        run_profile(args.profile, args.pin_sweeps, args.inner, args.n_up)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
