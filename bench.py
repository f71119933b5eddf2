#!/usr/bin/env python
"""Benchmark of the fast tensor-product Schwarz smoother library on one GB300.

Workload (one "step"): the additive vertex-patch Schwarz smoother (Alg. 2,
x = 0 form: x = omega sum_j R_j^T A_j^{-1} R_j b, fast diagonalization of
Sec. 3.2) on a 3D tensor grid of 32^3 cells with per-direction widths drawn
U[0.5, 1.5]/32 (seed 2), omega = 0.7, applied to 8 right-hand sides U[-1, 1]
(seeds 100..107) in one batched call, for each degree k = 2..7, in FP64.
Metric: DoF/s = sum over k of ndofs(k) * 8 per step / time per step.

Also reported: per-degree DoF/s and roofline fraction, an end-to-end number
through the same C-ABI call with host buffers (copies timed), the oracle on
the host cores as cpu_baseline, the MG-CG time to a 1e-8 residual
reduction on 64^3 cells (FP64 and mixed precision), batched solves, the
paper's fractional iteration counts, the k = 15 smoothers on the paper's
16^3-cell FLOP-table mesh, and the distorted meshes of Sec. 4 (2D and 3D:
mapped operators in FP64 and FP32, ACS / MCS sweeps with Cartesian-surrogate
cell solvers, V-cycle and PCG times with FP64 and FP32 V-cycles, the paper's
counts and its damping sweep).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tpss|reference]
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

NC = 32
KS = [2, 3, 4, 5, 6, 7]
SEEDS = list(range(100, 108))
OMEGA = 0.7
WIDTH_SEED = 2
METRIC = "patch-smoother DoF/s & MG-CG time-to-1e-8: mixed/batched vs FP64 plain, 1 GB300"
CONFIG = {"workload": "3D additive vertex-patch Schwarz smoother (fast diagonalization), 32^3 cells, "
                      "widths U[0.5,1.5]/32, omega 0.7, k=2..7, 8 RHS U[-1,1] batched, x=0 form",
          "cells": [NC, NC, NC], "degrees": KS, "nrhs": len(SEEDS),
          "l2": "inputs larger than L2 (each step streams >= 2.5 GB of vectors and tables)"}
# DRAM bytes (read + write) of one FP64 smoother call at k=7 (8 RHS) at the
# full 32^3 size, from a single-pass ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum over the call's launches; captured again after the
# kernel's last change, same value; taken with one launch per color, where
# the call now issues each color as two launches of 4 RHS on two streams,
# the same CTAs); set to None when the kernel changes after that capture.
TRAFFIC_K7_PER_CALL = 30.98e9


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="tpss", choices=["tpss", "reference"])
    p.add_argument("--no-mgcg", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--no-high-degree", action="store_true")
    p.add_argument("--no-kernels", action="store_true")
    p.add_argument("--no-distorted", action="store_true")
    p.add_argument("--batch-problems", type=int, default=48, help="use the first N problems of the batch (profiling)")
    p.add_argument("--batch-persistent", action="store_true",
                   help="also time the BF16 batch with every level in the persistent kernel")
    p.add_argument("--ks", default=",".join(map(str, KS)))
    p.add_argument("--nc", type=int, default=NC, help="cells per direction (profiling of small cases)")
    p.add_argument("--mixed", default="fp32,tf32,bf16", help="low-precision smoother variants to time")
    p.add_argument("--cpu-worker", type=int, default=0, help=argparse.SUPPRESS)
    return p.parse_args()


# --------------------------------------------------------------- ranks
def reduce_max(value, world, device):
    """Max over ranks of a host float (the timed region of the slowest rank);
    identity on one rank.  Works with NCCL (device cuda) and gloo (cpu)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank_step, steps, world, max_ms):
    """Whole-job throughput: units processed by all ranks / slowest rank's time."""
    return units_per_rank_step * steps * world / (max_ms / 1e3)


# ------------------------------------------------------------------ clocks
def clocks_start(path):
    fields = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={fields}", "--format=csv,noheader,nounits",
                                 "-lms", "200"], stdout=f, stderr=subprocess.DEVNULL), f
    except (OSError, FileNotFoundError):
        return None, None


def clocks_stop(proc, f, path, gpu_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
    f.close()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or parts[0] != str(gpu_index):
            continue
        try:
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
            "reasons": sorted(reasons)}


# -------------------------------------------------------------- cpu oracle
def cpu_model():
    """CPU model name of this host (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def fd_sample(ks, colors, threads):
    """Time the fast-diagonalization oracle (oracle/fd_smoother.c, FP64,
    OpenMP) on the bench workload restricted to the vertex patches of the
    given additive colors, 8 RHS, per degree.  Returns {k: (seconds, patches
    solved)}; the 1D eigendata are computed before the clock starts."""
    import numpy as np

    from oracle import fastdiag
    from paper_1910_11239_gb300 import workloads

    widths = workloads.widths_random(NC, 3, WIDTH_SEED)
    out = {}
    for k in ks:
        eig = fastdiag.eigendata(widths, k, True)
        b = workloads.rhs_batch(dofs(k), SEEDS)
        t0 = time.perf_counter()
        fastdiag.additive_local_sum(widths, k, True, b, OMEGA, nrhs=len(SEEDS), threads=threads, eig=eig,
                                    colors=colors)
        out[k] = (time.perf_counter() - t0, sum(fastdiag.count_color((NC, NC, NC), c) for c in colors))
    return out


def lu_sample(k, m, seed):
    """Time the dense-LU oracle (local matrices assembled from the bilinear
    form, LU with partial pivoting, one core) on m random vertex patches at
    degree k, 8 RHS; returns (seconds, m)."""
    import numpy as np
    import scipy.linalg as sla

    from oracle import schwarz
    from oracle.mesh import TensorMesh
    from oracle.sipg import SIPG
    from paper_1910_11239_gb300 import workloads

    mesh = TensorMesh(workloads.widths_random(NC, 3, WIDTH_SEED))
    patches = schwarz.vertex_patches(mesh)
    S = SIPG(mesh, k)
    pick = np.random.default_rng(seed).choice(len(patches), size=m, replace=False)
    N = mesh.num_cells * S.nloc
    b = workloads.rhs_batch(N, SEEDS).reshape(len(SEEDS), N)
    y = np.zeros_like(b)
    t0 = time.perf_counter()
    for j in pick:
        idx = schwarz.patch_dofs(patches[j][1], S.nloc)
        lu = sla.lu_factor(S.assemble(patches[j][1]).toarray())
        y[:, idx] += OMEGA * sla.lu_solve(lu, b[:, idx].T).T
    return time.perf_counter() - t0, m


def dofs(k):
    return NC ** 3 * (k + 1) ** 3


def npatches():
    return (NC - 1) ** 3


def sample_rate(per_k):
    """DoF/s of a sample: each degree contributes ndofs * 8 RHS scaled by the
    fraction of the patches solved, over the summed time."""
    work = sum(dofs(k) * len(SEEDS) * m / npatches() for k, (t, m) in per_k.items())
    return work / sum(t for t, _ in per_k.values())


def full_step_estimate_ms(per_k):
    """Time one whole step (every patch of every degree) would take at the
    sampled per-patch rate (reported beside the timed sample, never as it)."""
    return 1e3 * sum(t * npatches() / m for t, m in per_k.values())


CPU_COLORS = [0]             # one of the 8 additive colors: about 1/8 of the patches
CPU_ONE_CORE_KS = [2, 3, 4]  # the one-core run stays bounded
LU_K, LU_PATCHES = 2, 24     # dense LU (the non-tensor sACS approach), context only


def cpu_worker(ks):
    """The cpu_baseline measurement (run in a child process before any CUDA
    call): the fast-diagonalization oracle on all host cores and on one core,
    and the dense-LU oracle on one core, each on a bounded sample."""
    from oracle import fastdiag
    fastdiag.lib()
    fd_sample(ks[:1], CPU_COLORS, 0)   # warm-up (page in, thread pool)
    allc = fd_sample(ks, CPU_COLORS, 0)
    one_ks = [k for k in ks if k in CPU_ONE_CORE_KS] or ks[:1]
    one = fd_sample(one_ks, CPU_COLORS, 1)
    same = {k: allc[k] for k in one_ks}
    lu = {LU_K: lu_sample(LU_K, LU_PATCHES, 1000)}
    ncol = ", ".join(f"k={k}: {m}" for k, (t, m) in allc.items())
    return {
        "value": sample_rate(allc), "unit": "DoF/s", "cores": fastdiag.max_threads(), "kind": "oracle",
        "sample": (f"fast-diagonalization oracle (oracle/fd_smoother.c, FP64, OpenMP over the patches of one "
                   f"color), the vertex patches of additive color {CPU_COLORS} ({ncol} of {npatches()}), 8 RHS "
                   f"each; DoF/s = ndofs x 8 x solved/total patches / time"),
        "timed_s": sum(t for t, _ in allc.values()), "full_step_estimate_ms": full_step_estimate_ms(allc),
        "nproc": os.cpu_count(), "cpu_model": cpu_model(),
        "per_degree_s": {str(k): t for k, (t, _) in allc.items()},
        "one_core": {"value": sample_rate(one), "degrees": one_ks, "cores": 1,
                     "all_cores_same_degrees": sample_rate(same)},
        "dense_lu_one_core": {"value": sample_rate(lu), "degree": LU_K,
                              "sample": f"{LU_PATCHES} random vertex patches at k={LU_K}, 8 RHS"}}


def cpu_baseline_subprocess(ks):
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    env.pop("OMP_NUM_THREADS", None)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-worker", "1", "--ks", ",".join(map(str, ks))]
    res = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=900)
    if res.returncode != 0:
        return {"error": res.stderr[-400:]}
    return json.loads(res.stdout.strip().splitlines()[-1])


# --------------------------------------------------------------- reference
def run_reference(args):
    """The reference arm: the oracle (fast diagonalization in plain C with
    OpenMP on all host cores) on the same workload, each step a bounded sample
    (the vertex patches of one additive color, cycling through the 8 colors,
    at every degree).  ms_per_step is the timed interval of a step; value is
    the DoFs the sampled patches account for over that time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import fastdiag
    fastdiag.lib()
    ks = [int(x) for x in args.ks.split(",")]
    for w in range(args.warmup):
        fd_sample(ks, [w % 8], 0)
    steps = []
    for s in range(args.steps):
        steps.append(fd_sample(ks, [s % 8], 0))
    tot = {k: (sum(st[k][0] for st in steps), sum(st[k][1] for st in steps)) for k in ks}
    val = sample_rate(tot)
    step_ms = 1e3 * sum(t for t, _ in tot.values()) / max(1, args.steps)
    desc = (f"fast-diagonalization oracle (oracle/fd_smoother.c, FP64, OpenMP), per step the vertex patches of "
            f"one additive color (step s: color s mod 8, about 1/8 of {npatches()}) at k={ks[0]}..{ks[-1]}, 8 RHS")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "DoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": CONFIG,
            "full_step_estimate_ms": full_step_estimate_ms(tot),
            "cpu_baseline": {"value": val, "unit": "DoF/s", "cores": fastdiag.max_threads(), "kind": "oracle",
                             "sample": desc, "nproc": os.cpu_count(), "cpu_model": cpu_model()},
            "e2e": {"value": val, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ----------------------------------------------------------------- GPU arm
def main():
    global NC, BATCH_PROBLEMS
    args = parse()
    NC = args.nc
    BATCH_PROBLEMS = args.batch_problems
    if NC != 32:
        CONFIG["cells"] = [NC, NC, NC]
        CONFIG["workload"] = CONFIG["workload"].replace("32^3", f"{NC}^3").replace("/32", f"/{NC}")
    if args.cpu_worker:
        print(json.dumps(cpu_worker([int(x) for x in args.ks.split(",")])))
        return
    if args.impl == "reference":
        run_reference(args)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1910_11239_gb300 import perf, tpss, workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    ks = [int(x) for x in args.ks.split(",")]
    cpu_res = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_res = cpu_baseline_subprocess(ks)   # before the first CUDA call
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    widths = workloads.widths_random(NC, 3, WIDTH_SEED)
    stream = torch.cuda.current_stream()
    probs, pats, bdev, xdev, bhost, xhost = {}, {}, {}, {}, {}, {}
    for k in ks:
        probs[k] = tpss.Problem(3, k, widths, stream=stream)
        pats[k] = probs[k].setup_patches(0, tpss.VERTEX_PATCH)
        N = probs[k].ndofs(0)
        assert N == dofs(k)
        b = workloads.rhs_batch(N, SEEDS)
        bhost[k] = torch.from_numpy(b).pin_memory()
        xhost[k] = torch.empty_like(bhost[k]).pin_memory()
        bdev[k] = bhost[k].to("cuda")
        xdev[k] = torch.empty_like(bdev[k])
    nr = len(SEEDS)
    dofs_step = sum(dofs(k) * nr for k in ks)

    def step(evs=None):
        for k in ks:
            if evs is not None:
                evs[k][0].record()
            pats[k].smooth_additive(OMEGA, bdev[k], xdev[k], x_is_zero=True, nrhs=nr)
            if evs is not None:
                evs[k][1].record()

    nwarm = max(args.warmup, 3)
    for _ in range(nwarm):
        step()
    torch.cuda.synchronize()
    clk_path = f"/tmp/tpss_clocks_{os.getpid()}_{rank}.csv"
    cproc, cfile = clocks_start(clk_path)
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kev = [{k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for k in ks}
           for _ in range(args.steps)]
    e0.record()
    for s in range(args.steps):
        step(kev[s])
    e1.record()
    torch.cuda.synchronize()
    barrier()
    clocks = clocks_stop(cproc, cfile, clk_path, local)
    try:
        os.remove(clk_path)
    except OSError:
        pass
    ms = reduce_max(e0.elapsed_time(e1), world, "cuda")
    value = aggregate_rate(dofs_step, args.steps, world, ms)
    per_k = {}
    for k in ks:
        kms = statistics.mean(kev[s][k][0].elapsed_time(kev[s][k][1]) for s in range(args.steps))
        fl = perf.smoother_flops((NC, NC, NC), k, vertex=True, nrhs=nr)
        per_k[str(k)] = {"dofs_per_s": dofs(k) * nr / (kms / 1e3), "ms_per_call": kms,
                         "tflops": fl / (kms / 1e3) / 1e12,
                         "frac_fp64_peak": fl / (kms / 1e3) / perf.fp64_peak_flops()}
    kdom = max(ks, key=lambda k: per_k[str(k)]["ms_per_call"])
    dom = per_k[str(kdom)]
    roofline = {"bound": "alu", "kernel": f"patch_smooth_kernel<3,{2 * (kdom + 1)},vertex,double> (k={kdom})",
                "achieved": dom["tflops"], "peak": perf.fp64_peak_flops() / 1e12, "unit": "TFLOP/s",
                "frac": dom["frac_fp64_peak"],
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (FP64 pipe; HBM is not binding)",
                "per": "one smoother call = 8 colors x 2 halves of the 8 RHS (two streams) = 16 launches",
                "traffic": TRAFFIC_K7_PER_CALL if (kdom == 7 and NC == 32) else None,
                "traffic_unit": "bytes per call (dram read + write, ncu)",
                "algorithmic_bytes": perf.smoother_bytes((NC, NC, NC), kdom, nrhs=nr)}

    # end to end through the same call with host buffers (H2D + smooth + D2H),
    # the copies pipelined with the smoothing: the degrees of a step are
    # independent, so degree k+1's inputs are uploaded on one copy stream and
    # degree k-1's result is read back on another while degree k is smoothed.
    h2d = sum(bhost[k].numel() * 8 for k in ks)
    d2h = sum(xhost[k].numel() * 8 for k in ks)
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev = {name: {k: torch.cuda.Event() for k in ks} for name in ("in", "done", "out")}
    started = {k: False for k in ks}

    def e2e_step():
        for k in ks:
            with torch.cuda.stream(s_in):
                if started[k]:
                    s_in.wait_event(ev["done"][k])     # the previous step's smoother read bdev[k]
                bdev[k].copy_(bhost[k], non_blocking=True)
                ev["in"][k].record(s_in)
            stream.wait_event(ev["in"][k])
            if started[k]:
                stream.wait_event(ev["out"][k])        # the previous step's read-back of xdev[k]
            pats[k].smooth_additive(OMEGA, bdev[k], xdev[k], x_is_zero=True, nrhs=nr)
            ev["done"][k].record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev["done"][k])
                xhost[k].copy_(xdev[k], non_blocking=True)
                ev["out"][k].record(s_out)
            started[k] = True

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    s_in.wait_event(f0)   # no upload of the timed region starts before f0
    for _ in range(args.steps):
        e2e_step()
    for k in ks:
        stream.wait_event(ev["out"][k])   # the last read-backs are inside the timed region
    f1.record(stream)
    torch.cuda.synchronize()
    ems = reduce_max(f0.elapsed_time(f1), world, "cuda")
    e2e = {"value": aggregate_rate(dofs_step, args.steps, world, ems), "unit": "DoF/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "note": "pinned host buffers; uploads and read-backs on two copy streams overlap the smoothing of "
                   "the other degrees"}
    for k in ks:
        probs[k].close()
    del bdev, xdev, bhost, xhost

    def leg(name, fn):
        """Run one extra leg and print it as its own JSON line (rank 0)."""
        t0 = time.perf_counter()
        res = fn()
        if rank == 0:
            print(json.dumps({"leg": name, "wall_s": time.perf_counter() - t0, "result": res}), flush=True)

    for prec in [p for p in args.mixed.split(",") if p]:
        leg(f"mixed_smoother_{prec}",
            lambda: run_low_precision_smoother(prec, ks, widths, args.steps, tpss, workloads, perf, torch))
    if not args.no_mgcg:
        leg("mg_cg", lambda: run_mgcg(tpss, workloads, torch, MGCG_CASES))
        leg("paper_iterations", lambda: run_paper_iterations(tpss, workloads, perf, torch))
    if not args.no_batch:
        leg("batched", lambda: run_batch(tpss, workloads, perf, torch, args.steps, args.batch_persistent))
    if not args.no_kernels:
        leg("kernels", lambda: run_kernels(tpss, workloads, perf, torch, max(3, min(args.steps, 10))))
    if not args.no_high_degree:
        leg("high_degree_k15", lambda: run_high_degree(tpss, workloads, perf, torch, max(2, min(args.steps, 5))))
    if not args.no_distorted:
        leg("distorted", lambda: run_distorted(tpss, workloads, perf, torch, max(3, min(args.steps, 10))))

    if rank == 0:
        print(json.dumps(headline_line(value, ms / args.steps, world, args.steps, nwarm, roofline, e2e, clocks,
                                       per_k, cpu_res, args.steps * len(ks) * 8 * (2 if len(SEEDS) >= 2 else 1))),
              flush=True)
    if world > 1:
        dist.destroy_process_group()


def headline_line(value, ms_per_step, world, steps, warmup, roofline, e2e, clocks, per_k, cpu_res, launches):
    """The bench's contract line (printed last, a few KB): the FP64 smoother
    headline with its roofline, end-to-end number, clocks, per-degree rates
    and the CPU baseline.  The extra legs are printed on earlier lines."""
    line = {"impl": "tpss", "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded widths and right-hand sides)",
            "config": dict(CONFIG, parallelism=f"replicas x{world}") if world > 1 else CONFIG,
            "gpu_launches": launches, "roofline": roofline, "e2e": e2e, "clocks": clocks, "per_degree": per_k}
    if cpu_res is None:
        pass
    elif "value" in cpu_res:
        line["cpu_baseline"] = cpu_res
    else:
        line["cpu_baseline"] = {"value": None, "unit": "DoF/s", "cores": None, "kind": "oracle",
                                "sample": "failed: " + str(cpu_res.get("error", ""))[-300:]}
    return line


def run_low_precision_smoother(prec, ks, widths, steps, tpss, workloads, perf, torch):
    """The same smoother workload with FP32 vectors and FP32 / TF32 / BF16
    mode contractions (FP32 accumulation).  Roofline: HBM, 8 bytes per DoF
    and right-hand side (read b, write x) against the measured copy bandwidth."""
    import json as _json
    peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
    hbm = peaks.get("hbm_gbs", 6800.0)
    nr = len(SEEDS)
    out = {"dtype": prec, "accumulate": "fp32", "per_degree": {}}
    out["schedule"] = ("default: tcgen05 column streaming for k >= 4 (4 launches, r read and x written once per "
                       "parity class), colored launches for k <= 3; colored, plane-by-plane, atomic and both column "
                       "schedules timed beside it" if prec == "bf16"
                       else "default: tcgen05 column streaming (TF32 operands) for k >= 4, colored launches for "
                       "k <= 3; colored, plane-by-plane and tcgen05 schedules timed beside it" if prec == "tf32"
                       else "colored launches (default); plane-by-plane schedule timed beside it")
    total_ms = 0.0
    for k in ks:
        prob = tpss.Problem(3, k, widths)
        P = prob.setup_patches(0, tpss.VERTEX_PATCH, tpss.PRECISIONS[prec])
        N = prob.ndofs(0)
        b = torch.from_numpy(workloads.rhs_batch(N, SEEDS)).to("cuda", torch.float32)
        x = torch.empty_like(b)
        for _ in range(3):
            P.smooth_additive(OMEGA, b, x, x_is_zero=True, nrhs=nr)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            P.smooth_additive(OMEGA, b, x, x_is_zero=True, nrhs=nr)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        total_ms += ms
        byt = perf.smoother_bytes((NC, NC, NC), k, nrhs=nr, word=4)
        out["per_degree"][str(k)] = {"dofs_per_s": dofs(k) * nr / (ms / 1e3), "ms_per_call": ms,
                                     "hbm_gbs": byt / (ms / 1e3) / 1e9, "frac_hbm": byt / (ms / 1e3) / 1e9 / hbm}
        # the other schedules of the same smoother (default: column streaming
        # for BF16, colored launches otherwise)
        for name, sch in (("colors", tpss.ADDITIVE_COLORS), ("planes", tpss.ADDITIVE_PLANES),
                          ("atomic", tpss.ADDITIVE_ATOMIC), ("columns_mma_sync", tpss.ADDITIVE_COLUMNS),
                          ("columns_tcgen05", tpss.ADDITIVE_TCGEN05)):
            allowed = {"bf16": (tpss.ADDITIVE_COLORS, tpss.ADDITIVE_PLANES, tpss.ADDITIVE_ATOMIC,
                                tpss.ADDITIVE_COLUMNS, tpss.ADDITIVE_TCGEN05),
                       "tf32": (tpss.ADDITIVE_COLORS, tpss.ADDITIVE_PLANES, tpss.ADDITIVE_TCGEN05)}.get(
                           prec, (tpss.ADDITIVE_PLANES,))
            if sch not in allowed:
                continue
            P.set_additive_schedule(sch)
            P.smooth_additive(OMEGA, b, x, x_is_zero=True, nrhs=nr)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(steps):
                P.smooth_additive(OMEGA, b, x, x_is_zero=True, nrhs=nr)
            e1.record()
            torch.cuda.synchronize()
            out["per_degree"][str(k)][f"{name}_ms_per_call"] = e0.elapsed_time(e1) / steps
        prob.close()
    out["dofs_per_s"] = sum(dofs(k) * nr for k in ks) / (total_ms / 1e3)
    out["vs_fp64_note"] = "same workload, FP32 vectors; compare with the line's FP64 value"
    out["hbm_peak_gbs"] = hbm
    return out


def run_mgcg(tpss, workloads, torch, cases):
    """MG-CG on the unit cube, levels 2^3..64^3 cells, f = 3 pi^2 sin sin sin,
    V-cycle(1,1) preconditioned CG from x = 0 to a 1e-8 relative residual.
    For every (k, smoother, omega, precisions): time to solution (CUDA events
    around tpss_pcg_solve, setup excluded), iterations, and for the mixed
    precisions the relative difference to the FP64 solution.  Mixed runs use
    flexible CG with the FP32 V-cycle (FP32/TF32/BF16 mode contractions)."""
    out = {"workload": "3D unit cube, 2^3..64^3 cells (6 levels), f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z), "
                       "g = 0, rtol 1e-8; time excludes setup"}
    for k, sm, omega, precs in cases:
        prob = tpss.Problem(3, k, workloads.widths_uniform(2, 3), nlevels=6)
        N = prob.ndofs(5)
        b = torch.empty(N, dtype=torch.float64, device="cuda")
        prob.assemble_rhs(5, 0, b)
        x64 = torch.zeros_like(b)
        x = torch.empty_like(b)
        for prec_mode in precs:
            # "+full": Alg. 3 as printed (residual recomputed before every
            # color) instead of the default per-color residual update;
            # "+8colors": the 2^d-color vertex coloring (face-conflicting)
            prec = prec_mode.split("+")[0]
            full, colors8 = "+full" in prec_mode, "+8colors" in prec_mode
            prob.mg_setup(sm, omega, tpss.PRECISIONS[prec], flexible_cg=0 if prec == "fp64" else 1,
                          mult_residual=tpss.MULT_RESIDUAL_FULL if full else tpss.MULT_RESIDUAL_UPDATE,
                          mult_colors=8 if colors8 else 0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            try:
                res = prob.pcg_solve(b, x, rtol=1e-8, maxit=60)
                status = "converged" if res["converged"] else "not converged"
            except tpss.TpssError as e:
                res, status = {"iters": None, "rel_res": None}, str(e).split(":")[0]
            e1.record()
            torch.cuda.synchronize()
            rec = {"time_s": e0.elapsed_time(e1) / 1e3, "iterations": res["iters"], "rel_res": res["rel_res"],
                   "status": status, "ndofs": N}
            if prec_mode == "fp64" and status == "converged":
                x64.copy_(x)
            elif status == "converged" and x64.abs().max().item() > 0:
                rec["rel_diff_to_fp64_solution"] = ((x - x64).norm() / x64.norm()).item()
            if prec != "fp64" and not full and not colors8:
                # the same V-cycle inside mixed-precision iterative refinement
                torch.cuda.synchronize()
                e0.record()
                ir = prob.ir_solve(b, x, rtol=1e-8, inner_rtol=1e-3)
                e1.record()
                torch.cuda.synchronize()
                rec["iterative_refinement"] = {"time_s": e0.elapsed_time(e1) / 1e3, "outer": ir["outer"],
                                               "inner_iterations": ir["inner"], "rel_res": ir["rel_res"],
                                               "converged": ir["converged"]}
            out[f"k{k}_{sm}_omega{omega:g}_{prec}" + ("_full_residual_per_color" if full else "")
                + ("_8colors_face_conflicting" if colors8 else "")] = rec
        prob.close()
    return out


BATCH_PROBLEMS = 48

# Fractional iteration counts printed in the paper (tab:cubecp, tab:cubemvp),
# 3D, level L = 3 (16^3 cells), Gaussian-bell solution; ACS with CG, MCS and
# MVS with GMRES (reported here both with GMRES and the non-symmetric V-cycle,
# as in the paper, and with CG and the symmetric color order).
PAPER_NU = {("ACS", 3): 17.1, ("ACS", 7): 21.9, ("MCS", 3): 8.6, ("MCS", 7): 11.8, ("MVS", 3): 2.4, ("MVS", 7): 2.1}


def run_paper_iterations(tpss, workloads, perf, torch):
    """Fractional iterations on the paper's setup (unit cube, T_0 = 2^3 cells,
    L = 3, Gaussian bells with boundary data, V-cycle(1,1), rtol 1e-8), next
    to the paper's values: ACS with CG (residual-based and, as the paper
    measures CG, energy-norm based), MCS / MVS with CG and the symmetric
    color order, and with GMRES and the non-symmetric V-cycle (right and left
    preconditioning).  Coarse solve exact (the Chebyshev coarse solver gives
    the same counts, tests/test_gpu_chebyshev.py)."""
    out = {}
    for k in (3, 7):
        prob = tpss.Problem(3, k, workloads.widths_uniform(2, 3), nlevels=4)
        N = prob.ndofs(3)
        b = torch.empty(N, dtype=torch.float64, device="cuda")
        prob.assemble_rhs(3, 1, b)
        x = torch.empty_like(b)
        for sm, omega in (("ACS", 0.7), ("MCS", 1.0), ("MVS", 1.0)):
            prob.mg_setup(sm, omega, tpss.FP64)
            res = prob.pcg_solve(b, x, rtol=1e-8, maxit=100, history=True)
            out[f"{sm}_k{k}_cg"] = {"iterations": res["iters"],
                                    "nu_frac_residual": perf.fractional_iterations(res["history"], 1e-8),
                                    "paper_nu_frac": PAPER_NU[(sm, k)]}
            if sm == "ACS":   # the paper's CG measure: energy norm of the error
                out[f"{sm}_k{k}_cg"]["nu_frac_energy"] = perf.fractional_iterations(
                    perf.cg_energy_errors(prob, b), 1e-8)
            if sm != "ACS":   # the paper's method for multiplicative smoothers: GMRES, non-symmetric V-cycle
                prob.mg_setup(sm, omega, tpss.FP64, nonsymmetric=1)
                for left in (False, True):   # right / left preconditioning (the paper does not say)
                    res = prob.gmres_solve(b, x, rtol=1e-8, maxit=100, restart=30, history=True, left=left)
                    out[f"{sm}_k{k}_gmres" + ("_left" if left else "")] = {
                        "iterations": res["iters"],
                        "nu_frac_residual": perf.fractional_iterations(res["history"], 1e-8),
                        "paper_nu_frac": PAPER_NU[(sm, k)]}
        prob.close()
    return out


def _time_calls(torch, fn, steps):
    """Mean milliseconds of fn() over `steps` calls after 2 warm-up calls,
    CUDA events on the current stream."""
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_kernels(tpss, workloads, perf, torch, steps):
    """The other kernels of the path on 32^3 cells (fine level of a 16^3 ->
    32^3 pair, widths U[0.5,1.5] per cell): the matrix-free operator (FP64
    and FP32), the transfers, and one multiplicative vertex-patch sweep with
    the residual updated per color and recomputed per color; each with its
    algorithmic flops and bytes against the FP64 pipe, FP32 pipe or HBM peak."""
    import json as _json
    peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
    hbm = peaks.get("hbm_gbs", 6800.0)
    out = {"workload": "3D, 32^3 cells (fine level of 16^3 -> 32^3), widths U[0.5,1.5]/16 (seed 2), 1 RHS",
           "peaks": {"fp64_tflops": perf.fp64_peak_flops() / 1e12, "fp32_tflops": perf.fp32_peak_flops() / 1e12,
                     "hbm_gbs": hbm}}
    cw = workloads.widths_random(16, 3, WIDTH_SEED)
    fine, coarse = (32, 32, 32), (16, 16, 16)
    for k in (4, 7):
        prob = tpss.Problem(3, k, cw, nlevels=2)
        nf, nc = prob.ndofs(1), prob.ndofs(0)
        u = torch.from_numpy(workloads.rhs_uniform(nf, seed=3)).to("cuda")
        au = torch.empty_like(u)
        rec = {}
        ms = _time_calls(torch, lambda: prob.apply_operator(1, u, au), steps)
        fl, by = perf.operator_flops(fine, k), perf.operator_bytes(fine, k)
        rec["operator_fp64"] = {"ms": ms, "tflops": fl / ms / 1e9, "frac_fp64_peak": fl / ms / 1e9 / (
            perf.fp64_peak_flops() / 1e12), "algorithmic_gbs": by / ms / 1e6}
        u32, au32 = u.float(), torch.empty(nf, dtype=torch.float32, device="cuda")
        ms = _time_calls(torch, lambda: prob.apply_operator(1, u32, au32), steps)
        by32 = perf.operator_bytes(fine, k, word=4)
        rec["operator_fp32"] = {"ms": ms, "tflops": fl / ms / 1e9,
                                "frac_fp32_peak": fl / ms / 1e9 / (perf.fp32_peak_flops() / 1e12),
                                "algorithmic_gbs": by32 / ms / 1e6, "frac_hbm": by32 / ms / 1e6 / hbm,
                                "note": "three sum-factorization passes stream 4 intermediate vectors through HBM"}
        c = torch.from_numpy(workloads.rhs_uniform(nc, seed=4)).to("cuda")
        ms = _time_calls(torch, lambda: prob.prolongate_add(1, c, au), steps)
        fl = perf.transfer_flops(coarse, k)
        by = perf.transfer_bytes(coarse, k, prolong=True)
        rec["prolongate_add_fp64"] = {"ms": ms, "tflops": fl / ms / 1e9,
                                      "frac_fp64_peak": fl / ms / 1e9 / (perf.fp64_peak_flops() / 1e12),
                                      "algorithmic_gbs": by / ms / 1e6}
        ms = _time_calls(torch, lambda: prob.restrict(1, u, c), steps)
        by = perf.transfer_bytes(coarse, k, prolong=False)
        rec["restrict_fp64"] = {"ms": ms, "tflops": fl / ms / 1e9,
                                "frac_fp64_peak": fl / ms / 1e9 / (perf.fp64_peak_flops() / 1e12),
                                "algorithmic_gbs": by / ms / 1e6}
        P = prob.setup_patches(1, tpss.VERTEX_PATCH)
        x = torch.zeros_like(u)
        for mode, name in ((tpss.MULT_RESIDUAL_UPDATE, "mvs_sweep_fp64_residual_updated"),
                           (tpss.MULT_RESIDUAL_FULL, "mvs_sweep_fp64_residual_recomputed")):
            P.set_mult_residual(mode)
            ms = _time_calls(torch, lambda: P.smooth_multiplicative(1.0, u, x), max(2, steps // 2))
            rec[name] = {"ms": ms, "colors": 16}
        P.close()
        prob.close()
        out[f"k{k}"] = rec
    return out


# tab:flop-additive: MFLOP of all local solvers of one additive smoother
# application on T_3 = 16^3 cells (3375 vertex patches), d = 3, k = 15
PAPER_MFLOP_K15 = {"AVS": 42709, "ACS": 3256}
# tab:cubecp / tab:cubemvpminimal, 3D, L = 1, k = 15
PAPER_NU_K15_L1 = {"ACS": 28.5, "MCS": 15.7, "MVS": 1.5}


def run_high_degree(tpss, workloads, perf, torch, steps):
    """k = 15 in FP64 (subdomains of n = 32 points per direction): the
    additive vertex-patch and cell smoothers on the 16^3-cell mesh of the
    paper's local-solver FLOP table, timed per call (CUDA events), with the
    FLOP count of that table and the fraction of the FP64 pipe peak; and the
    residual-based fractional iterations of the k = 15 columns on 3D L = 1."""
    nc = 16
    widths = workloads.widths_random(nc, 3, WIDTH_SEED)
    out = {"workload": f"3D, {nc}^3 cells, widths U[0.5,1.5]/{nc} (seed {WIDTH_SEED}), k = 15, FP64, "
                       "1 RHS U[-1,1], x = 0 form"}
    prob = tpss.Problem(3, 15, widths)
    N = prob.ndofs(0)
    b = torch.from_numpy(workloads.rhs_batch(N, SEEDS[:1])).to("cuda")
    x = torch.empty_like(b)
    for name, kind, omega, kern in (("AVS", tpss.VERTEX_PATCH, 0.125, "patch_smooth_large_kernel<32>"),
                                    ("ACS", tpss.CELL, 0.7, "patch_smooth_kernel<3,16,cell,double>")):
        P = prob.setup_patches(0, kind)
        for _ in range(2):
            P.smooth_additive(omega, b, x, x_is_zero=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            P.smooth_additive(omega, b, x, x_is_zero=True)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        fl = perf.smoother_flops((nc, nc, nc), 15, vertex=kind == tpss.VERTEX_PATCH)
        out[name] = {"kernel": kern, "ms_per_call": ms, "mflop_per_call": fl / 1e6,
                     "paper_mflop_per_call": PAPER_MFLOP_K15[name], "tflops": fl / (ms / 1e3) / 1e12,
                     "frac_fp64_peak": fl / (ms / 1e3) / perf.fp64_peak_flops(),
                     "dofs_per_s": N / (ms / 1e3)}
        P.close()
    prob.close()
    its = {}
    prob = tpss.Problem(3, 15, workloads.widths_uniform(2, 3), nlevels=2)
    N = prob.ndofs(1)
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    prob.assemble_rhs(1, 1, b)
    x = torch.empty_like(b)
    for sm in ("ACS", "MCS", "MVS"):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if sm == "ACS":
            prob.mg_setup("ACS", 0.7, tpss.FP64)
            e0.record()
            res = prob.pcg_solve(b, x, rtol=1e-8, maxit=100, history=True)
        else:   # MCS: left preconditioning (reproduces the printed counts); MVS: right
            prob.mg_setup(sm, 1.0, tpss.FP64, nonsymmetric=1)
            e0.record()
            res = prob.gmres_solve(b, x, rtol=1e-8, maxit=100, restart=30, history=True, left=sm == "MCS")
        e1.record()
        torch.cuda.synchronize()
        its[f"{sm}_L1"] = {"krylov": {"ACS": "cg", "MCS": "gmres_left", "MVS": "gmres"}[sm], "iterations": res["iters"],
                           "nu_frac_residual": perf.fractional_iterations(res["history"], 1e-8),
                           "paper_nu_frac": PAPER_NU_K15_L1[sm], "time_s": e0.elapsed_time(e1) / 1e3}
    prob.close()
    out["paper_iterations_k15"] = its
    return out


# tab:cubedist25acp / tab:cubedist25mcp: (smoother, m, k) -> printed nu_frac;
# 2D at L = 3 (32 x 32 coarse cells), 3D at L = 1 (8^3 coarse cells), 25% distortion
PAPER_NU_DIST = {2: {("ACS", 1, 3): 38.7, ("ACS", 2, 3): 24.3, ("MCS", 1, 3): 24.7, ("MCS", 2, 3): 15.3,
                     ("ACS", 1, 7): 47.7, ("MCS", 1, 7): 43.5, ("ACS", 1, 15): 65.6, ("MCS", 1, 15): 50.9},
                 3: {("ACS", 1, 3): 34.4, ("ACS", 2, 3): 24.5, ("MCS", 1, 3): 24.7, ("MCS", 2, 3): 14.4,
                     ("ACS", 1, 7): 49.7, ("MCS", 1, 7): 37.7}}
# relaxation of those columns: ACS (k = 3, 7), MCS (k = 3, 7)
PAPER_OMEGA_DIST = {2: {("ACS", 3): 0.5, ("ACS", 7): 0.5, ("MCS", 3): 0.75, ("MCS", 7): 0.5, ("ACS", 15): 0.5,
                        ("MCS", 15): 0.5},
                    3: {("ACS", 3): 0.55, ("ACS", 7): 0.5, ("MCS", 3): 0.95, ("MCS", 7): 0.7}}
DIST_SEED = 1


def run_distorted(tpss, workloads, perf, torch, steps):
    """Sec. 4: the unit square (32^2 cells) / cube (8^3 cells) with 25% vertex
    distortion (seed DIST_SEED), gamma_hat = 4, refined to about 16.8 M DoFs
    (2D k = 3: L = 5; k = 7: L = 4; 3D k = 3: L = 3; k = 7: L = 2): the
    matrix-free operator, one ACS and one MCS sweep with Cartesian-surrogate
    cell solvers, the V-cycle and PCG to 1e-8 (f = d pi^2 prod sin(pi x_t),
    Chebyshev coarse solve), timed with CUDA events; and the energy-norm
    fractional counts of the paper's columns (2D L = 3, 3D L = 1)."""
    out = {"workload": f"unit square 32^2 / cube 8^3 coarse cells, 25% distortion (seed {DIST_SEED}), "
                       "gamma_hat 4, FP64"}
    fp64 = perf.fp64_peak_flops()
    peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
    HBM_GBS = json.load(open(peaks)).get("hbm_gbs", 6800.0) if os.path.exists(peaks) else 6800.0
    for dim, n0, runs, Lp in ((2, 32, ((3, 5), (7, 4)), 3), (3, 8, ((3, 3), (7, 2)), 1)):
        V0 = workloads.vertices_distorted(n0, DIST_SEED, dim=dim)
        rec_d = {}
        for k, L in runs:
            om_a, om_m = PAPER_OMEGA_DIST[dim][("ACS", k)], PAPER_OMEGA_DIST[dim][("MCS", k)]
            prob = tpss.Problem.mapped(k, V0, nlevels=L + 1, gamma_hat=4.0)
            N, nc = prob.level_info(L)
            u = torch.from_numpy(workloads.rhs_uniform(N, seed=3)).to("cuda")
            au = torch.empty_like(u)
            ms = _time_calls(torch, lambda: prob.apply_operator(L, u, au), steps)
            fl = (perf.mapped_operator_flops(nc[:2], k) if dim == 2 else perf.mapped3_operator_flops(nc, k))
            by = (perf.mapped_operator_bytes(nc[:2], k) if dim == 2 else perf.mapped3_operator_bytes(nc, k))
            rec = {"L": L, "cells": nc[0] * nc[1] * (nc[2] if dim == 3 else 1), "dofs": N,
                   "operator": {"kernel": f"mapped{'' if dim == 2 else '3'}_op_kernel<{k + 1}>", "ms": ms,
                                "dofs_per_s": N / (ms / 1e3), "tflops": fl / ms / 1e9,
                                "frac_fp64_peak": fl / (ms / 1e3) / fp64, "algorithmic_gbs": by / ms / 1e6}}
            u32, au32 = u.float(), torch.empty(N, dtype=torch.float32, device="cuda")
            ms32 = _time_calls(torch, lambda: prob.apply_operator(L, u32, au32), steps)
            by32 = (perf.mapped_operator_bytes(nc[:2], k, word=4) if dim == 2
                    else perf.mapped3_operator_bytes(nc, k, word=4))
            rec["operator_fp32"] = {"ms": ms32, "dofs_per_s": N / (ms32 / 1e3), "tflops": fl / ms32 / 1e9,
                                    "frac_fp32_peak": fl / (ms32 / 1e3) / perf.fp32_peak_flops(),
                                    "algorithmic_gbs": by32 / ms32 / 1e6, "frac_hbm": by32 / ms32 / 1e6 / HBM_GBS}
            b = torch.empty(N, dtype=torch.float64, device="cuda")
            prob.assemble_rhs(L, 0, b)
            x = torch.zeros_like(b)
            P = prob.setup_patches(L, tpss.CELL)
            ms = _time_calls(torch, lambda: P.smooth_additive(om_a, b, x, x_is_zero=True), steps)
            rec["acs_sweep_x0"] = {"ms": ms, "dofs_per_s": N / (ms / 1e3), "note": "x = 0: local solves only"}
            ms = _time_calls(torch, lambda: P.smooth_multiplicative(om_m, b, x), max(2, steps // 2))
            rec["mcs_sweep"] = {"ms": ms, "dofs_per_s": N / (ms / 1e3), "note": "2 colors, full residual per color"}
            P.close()
            for sm, om in (("ACS", om_a), ("MCS", om_m)):
                prob.mg_setup(sm, om, tpss.FP64, coarse_solver=tpss.COARSE_CHEBYSHEV)
                z = torch.empty_like(b)
                ms = _time_calls(torch, lambda: prob.vcycle(b, z), max(2, steps // 2))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                res = prob.pcg_solve(b, x, rtol=1e-8, maxit=200, history=True)
                e1.record()
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1) / 1e3
                rec[f"{sm}1_pcg"] = {"omega": om, "vcycle_ms": ms, "iterations": res["iters"],
                                     "nu_frac_residual": perf.fractional_iterations(res["history"], 1e-8),
                                     "solve_s": t, "dofs_per_s": N / t}
                # the same solve with the FP32 V-cycle (flexible PCG in FP64)
                prob.mg_setup(sm, om, tpss.FP32, flexible_cg=1, coarse_solver=tpss.COARSE_CHEBYSHEV)
                z = torch.empty_like(b)
                ms32 = _time_calls(torch, lambda: prob.vcycle(b, z), max(2, steps // 2))
                e0.record()
                res32 = prob.pcg_solve(b, x, rtol=1e-8, maxit=200)
                e1.record()
                torch.cuda.synchronize()
                t32 = e0.elapsed_time(e1) / 1e3
                rec[f"{sm}1_pcg_fp32_vcycle"] = {"vcycle_ms": ms32, "iterations": res32["iters"], "solve_s": t32,
                                                 "dofs_per_s": N / t32, "speedup_vs_fp64": t / t32}
                prob.mg_setup(sm, om, tpss.FP64, coarse_solver=tpss.COARSE_CHEBYSHEV)
                if sm == "ACS":   # the coarse solve's share of the V-cycle (Chebyshev, CUDA graph)
                    b0 = torch.from_numpy(workloads.rhs_uniform(prob.ndofs(0), seed=5)).to("cuda")
                    x0 = torch.empty_like(b0)
                    rec["coarse_solve"] = {"ms": _time_calls(torch, lambda: prob.coarse_solve(b0, x0), 3),
                                           "dofs": prob.ndofs(0), **prob.coarse_chebyshev_info()}
            prob.close()
            rec_d[f"k{k}"] = rec
        its = {}
        for (sm, m, k), paper in PAPER_NU_DIST[dim].items():
            om = PAPER_OMEGA_DIST[dim][(sm, k)]
            prob = tpss.Problem.mapped(k, V0, nlevels=Lp + 1, gamma_hat=4.0)
            prob.mg_setup(sm, om, tpss.FP64, coarse_solver=tpss.COARSE_CHEBYSHEV, smoothing_steps=m)
            b = torch.empty(prob.ndofs(Lp), dtype=torch.float64, device="cuda")
            prob.assemble_rhs(Lp, 0, b)
            errs = perf.cg_energy_errors(prob, b, rtol=1e-8, maxit=150)
            prob.close()
            its[f"{sm}{m}_k{k}_L{Lp}"] = {"omega": om, "nu_frac_energy": perf.fractional_iterations(errs, 1e-8),
                                          "paper_nu_frac": paper}
        rec_d[f"paper_iterations_L{Lp}"] = its
        if dim == 2:   # tab:cubedist25varydamp: k = 3, L = 3, one smoothing step, omega swept
            sweep = {}
            prob = tpss.Problem.mapped(3, V0, nlevels=4, gamma_hat=4.0)
            b = torch.empty(prob.ndofs(3), dtype=torch.float64, device="cuda")
            prob.assemble_rhs(3, 0, b)
            xs, xw = torch.empty_like(b), torch.empty_like(b)
            prob.mg_setup("ACS", 0.5, tpss.FP64, coarse_solver=tpss.COARSE_CHEBYSHEV)
            prob.pcg_solve(b, xs, rtol=1e-14, maxit=300)   # x* once, with a convergent V-cycle
            for sm, omegas, paper in (("ACS", (0.65, 0.6, 0.55, 0.5, 0.45, 0.4), (">100", 54.4, 40.7, 38.7, 42.9, 48.6)),
                                      ("MCS", (0.85, 0.8, 0.75, 0.7, 0.65, 0.6), (23.4, 23.6, 24.7, 25.8, 27.6, 29.6))):
                for om, pv in zip(omegas, paper):
                    prob.mg_setup(sm, om, tpss.FP64, coarse_solver=tpss.COARSE_CHEBYSHEV)
                    try:
                        errs = prob.pcg_energy_errors(b, xs, xw, rtol=1e-8, maxit=150)
                    except tpss.TpssError:
                        errs = [1.0, 1.0]
                    ok = errs[-1] <= 1e-8 * errs[0]
                    sweep[f"{sm}_w{om:.2f}"] = {"nu_frac_energy": perf.fractional_iterations(errs, 1e-8) if ok
                                                else ">150", "paper_nu_frac": pv}
            prob.close()
            rec_d["damping_sweep_k3_L3"] = sweep
        out[f"{dim}d"] = rec_d
    return out


def batch_specs(workloads):
    """48 problems = 12 each of (16^3, k=7), (24^3, k=5), (32^3, k=3), (48^3, k=2):
    coarse widths U[0.5,1.5] h (seed 1000+p), bisected; 4 RHS U[-1,1] (seed 2000+4p+r)."""
    kinds = [(16, 7, 2), (24, 5, 3), (32, 3, 2), (48, 2, 3)]
    out = []
    for p in range(48):
        n, k, c0 = kinds[p % 4]
        nl = 1
        while c0 << (nl - 1) < n:
            nl += 1
        out.append((k, workloads.widths_random(c0, 3, 1000 + p), nl))
    return out[:BATCH_PROBLEMS]


def run_batch(tpss, workloads, perf, torch, steps, persistent_too=False):
    """Config 5 in BF16 (per-problem smoothers on side streams; with
    persistent_too also with every level in the persistent kernel) and FP32
    (persistent kernel), then the same problems one at a time in FP64."""
    import numpy as np
    out = {"workload": "48 independent 3D Poisson problems, 12 each of (16^3,k=7), (24^3,k=5), (32^3,k=3), "
                       "(48^3,k=2), random widths, 4 RHS each U[-1,1]; AVS omega 1/8; FP32 V-cycle with one "
                       "persistent smoother launch per level (BF16: every level on the per-problem smoothers, "
                       "tcgen05 columns for k >= 4 and colored launches below, on 4 side streams; "
                       "bf16_persistent: every problem in the persistent kernel), per-problem operators and "
                       "transfers on the side streams, CUDA graph, FP64 flexible PCG to 1e-8"}
    variants = [("bf16", "bf16", True)] + ([("bf16", "bf16_persistent", False)] if persistent_too else []) + \
        [("fp32", "fp32", True)]
    for prec, key, columns in variants:
        out[key] = run_batch_one(tpss, workloads, torch, steps, prec, columns)
    specs = batch_specs(workloads)
    side = torch.cuda.Stream()
    nrhs = 4
    with torch.cuda.stream(side):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # one-at-a-time FP64 on the same problems (first right-hand side of each, x 4)
        t_fp64, its = 0.0, []
        for p, (k, widths, nl) in enumerate(specs):
            prob = tpss.Problem(3, k, widths, nlevels=nl, stream=side)
            prob.mg_setup("AVS", 0.125, tpss.FP64)
            n = prob.ndofs(nl - 1)
            bp = torch.from_numpy(workloads.rhs_uniform(n, 2000 + 4 * p)).to("cuda")
            xp = torch.empty_like(bp)
            torch.cuda.synchronize()
            e0.record(side)
            r = prob.pcg_solve(bp, xp, rtol=1e-8, maxit=100)
            e1.record(side)
            torch.cuda.synchronize()
            t_fp64 += e0.elapsed_time(e1) / 1e3
            its.append(r["iters"])
            prob.close()
        out["one_at_a_time_fp64"] = {"time_s": t_fp64 * nrhs,
                                     "measured": f"{len(specs)} problems x 1 RHS, times 4",
                                     "iters_max": int(max(its)), "iters_mean": float(np.mean(its))}
    for _, key, _ in variants:
        out[key]["speedup_time_to_solution_vs_fp64_one_at_a_time"] = (
            out["one_at_a_time_fp64"]["time_s"] / out[key]["pcg"]["time_s"])
    return out


def run_batch_one(tpss, workloads, torch, steps, prec, columns=True):
    import numpy as np
    specs = batch_specs(workloads)
    nrhs = 4
    side = torch.cuda.Stream()
    out = {"precision": prec, "columns": bool(columns and prec == "bf16")}
    with torch.cuda.stream(side):
        t0 = time.perf_counter()
        B = tpss.Batch(specs, nrhs=nrhs, omega=0.125, stream=side, precision=tpss.PRECISIONS[prec],
                       columns=columns)
        torch.cuda.synchronize()
        out["setup_s"] = time.perf_counter() - t0
        out["uses_graph"] = B.uses_graph
        out["ppb"] = {str(specs[p][0]): B.info(p)["ppb"] for p in range(4)}
        b = np.empty(B.total)
        ndofs = []
        for p in range(len(specs)):
            info = B.info(p)
            ndofs.append(info["ndofs"])
            for r in range(nrhs):
                o = info["offset"] + r * info["ndofs"]
                b[o:o + info["ndofs"]] = workloads.rhs_uniform(info["ndofs"], 2000 + 4 * p + r)
        out["total_dofs"] = int(sum(ndofs))
        b32 = torch.from_numpy(b).to("cuda", torch.float32)
        x32 = torch.empty_like(b32)
        for _ in range(3):
            B.smooth_additive(b32, x32)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(side)
        for _ in range(steps):
            B.smooth_additive(b32, x32)
        e1.record(side)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        byt = 8.0 * B.total
        peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
        hbm = json.load(open(peaks)).get("hbm_gbs", 6800.0) if os.path.exists(peaks) else 6800.0
        # BF16 with columns: every problem's finest level on its own passes (8 launches: 4 classes x 2
        # RHS halves of the tcgen05 columns for k >= 4, 8 colors below), none left for the persistent kernel
        out["smoother"] = {"dofs_per_s": B.total / (ms / 1e3), "ms_per_call": ms,
                           "launches_per_call": 8 * len(specs) if out["columns"] else 1,
                           "hbm_gbs": byt / (ms / 1e3) / 1e9, "frac_hbm": byt / (ms / 1e3) / 1e9 / hbm}
        bd = torch.from_numpy(b).to("cuda")
        x = torch.empty_like(bd)
        B.vcycle(bd, x)
        torch.cuda.synchronize()
        e0.record(side)
        for _ in range(steps):
            B.vcycle(bd, x)
        e1.record(side)
        torch.cuda.synchronize()
        out["vcycle_ms"] = e0.elapsed_time(e1) / steps
        e0.record(side)
        res = B.pcg_solve(bd, x, rtol=1e-8, maxit=100)
        e1.record(side)
        torch.cuda.synchronize()
        out["pcg"] = {"time_s": e0.elapsed_time(e1) / 1e3, "converged": bool(res["converged"]),
                      "iters_max": int(res["iters"].max()), "iters_mean": float(res["iters"].mean()),
                      "rel_res_max": float(res["rel_res"].max())}
        B.close()
    return out


MGCG_CASES = [
    (4, "AVS", 0.7, ["fp64"]),
    (4, "AVS", 0.125, ["fp64", "fp32", "tf32", "bf16"]),
    (4, "MVS", 1.0, ["fp64", "fp64+full", "fp64+8colors", "fp32", "tf32", "bf16"]),
    (3, "MVS", 1.0, ["fp64", "fp32", "tf32", "bf16"]),
    (5, "MVS", 1.0, ["fp64", "fp32", "tf32", "bf16"]),
    (7, "MVS", 1.0, ["fp64", "fp64+full", "fp32", "tf32", "bf16"]),
    (3, "AVS", 0.125, ["fp64", "fp32", "bf16"]),
    (5, "AVS", 0.125, ["fp64", "fp32", "bf16"]),
    (7, "AVS", 0.125, ["fp64", "fp32", "bf16"]),
]


if __name__ == "__main__":
    main()
