#!/usr/bin/env python3
"""Benchmark of the GMG-PCG Poisson solve (one JSON line on rank 0).

Workload (a "step"): one FP64 solve of -Laplace(u) = f, f = 3 pi^2 sin(pi x)
sin(pi y) sin(pi z), homogeneous Dirichlet BCs, P2 Lagrange on UnitCubeMesh
64^3 (1,572,864 cells, 129^3 = 2,146,689 dofs) built as a 4-level hierarchy
from an 8^3 mesh, CG preconditioned by one GMG V-cycle (2 Chebyshev-Jacobi
steps per level, FP64 Cholesky coarse solve), to ||r|| <= 1e-8 ||b||.  The
hierarchy and operator setup happen once before timing (as a solver object is
reused across right-hand sides).  Metric: solved DoF/s (all (2N+1)^3 dofs)
per step; steps are timed with CUDA events on the solve's stream, with L2
flushed between steps.

--impl reference times the CPU FP64 oracle (assembled CSR + GMG-PCG) on the
host cores on a bounded sample of the same workload (P2 UnitCubeMesh 32^3,
3 levels, same f and rtol), since the paper ships no runnable code.

Multi-GPU (torchrun, N>1): the solve does not shard in this build; every rank
solves its own replica (weak scaling, no collective on the data path).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {"workload": "poisson_p2_unitcube64_gmg4_fp64", "mesh": "UnitCubeMesh(64,64,64) Kuhn 6-tet",
            "degree": 2, "levels": 4, "coarse_mesh": 8, "cells": 1572864, "dofs": 2146689, "rtol": 1e-8,
            "preconditioner": "GMG V(2,2) Chebyshev-Jacobi + FP64 Cholesky coarse", "l2_between_steps": "flushed"}
SAMPLE = {"N0": 8, "nrefine": 2, "degree": 2}  # oracle bounded sample: P2 32^3, 3 levels
# FP64 flops of one P2 element application in the matrix-free kernel (c, d, S,
# four G-products, transpose: see the element routine), per tet.
FLOPS_PER_CELL_P2 = 160
FP64_PEAK_TFLOPS = 1.25  # GB300 nominal FP64 (152 SMs x 2.07 GHz x 2 FP64 FMA/clk/SM x 2)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        rows = [r.split(",") for r in open(self.file.name).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "samples": len(rows),
                "reasons": reasons}


# ------------------------------------------------------------ cpu oracle
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import fe_oracle as O
import fe_inputs as I
N0, nref, k, steps = {N0}, {nref}, {k}, {steps}
t0 = time.time()
h = O.Hierarchy(N0, nref, k)
L = h.fine
b = O.load_vector(L, I.sin_product_rhs(L.space.coords))
setup = time.time() - t0
times, its = [], []
for s in range(steps):
    t = time.time()
    u, it, hist = O.solve(h, b, rtol=1e-8)
    times.append(time.time() - t)
    its.append(it)
print(json.dumps({{"n": int(L.n), "setup_s": setup, "times": times, "iterations": its, "rel_res": hist[-1]}}))
"""


def run_oracle(steps):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET.format(root=ROOT, N0=SAMPLE["N0"], nref=SAMPLE["nrefine"], k=SAMPLE["degree"], steps=steps)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def sample_desc(r):
    return (f"oracle GMG-PCG solve (assembled CSR, scipy SpMV) of the same problem on P2 UnitCubeMesh "
            f"{SAMPLE['N0'] << SAMPLE['nrefine']}^3 ({r['n']} dofs, {SAMPLE['nrefine'] + 1} levels), rtol 1e-8, "
            f"{len(r['times'])} solve(s), setup {r['setup_s']:.1f}s excluded")


# --------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import fe_inputs as I
    from paper_2104_08012_gb300 import build as _build
    _build.build()
    import paper_2104_08012_gb300 as fe

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    t_setup = time.time()
    h = fe.Hierarchy(WORKLOAD["coarse_mesh"], WORKLOAD["levels"] - 1, WORKLOAD["degree"])
    n, C = h.n_dofs(), h.n_cells()
    assert n == WORKLOAD["dofs"] and C == WORKLOAD["cells"]
    f_host = I.sin_product_rhs(h.dof_coordinates())
    setup_s = time.time() - t_setup
    f = torch.from_numpy(f_host).to(dev)
    u = torch.empty(n, dtype=torch.float64, device=dev)
    opts = fe.default_opts(rtol=WORKLOAD["rtol"], profile=1)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)

    def step(rhs, out):
        return h.solve(rhs, out, opts=opts, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(f, u)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    launches0 = fe.fe_kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    torch.cuda.nvtx.range_push("timed")
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            ev[k][0].record(stream)
            stats.append(step(f, u))
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    launches = fe.fe_kernel_launches() - launches0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    # end-to-end: pinned host f in, host u out, through the C ABI (copies inside the timed region)
    f_pin = torch.from_numpy(f_host).pin_memory()
    u_pin = torch.empty(n, dtype=torch.float64).pin_memory()
    eve = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            eve[k][0].record(stream)
            step(f_pin, u_pin)
            eve[k][1].record(stream)
    torch.cuda.synchronize()
    te_ms = sum(a.elapsed_time(b) for a, b in eve)
    # correctness of the last solve: relative residual reported by the FP64 recurrence and an
    # independent check of the error against the analytic solution at the nodes
    u_host = u.cpu().numpy()
    nodal_err = float(np.abs(u_host - I.sin_product(h.dof_coordinates())).max())
    if world > 1:
        t = torch.tensor([t_ms, te_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_ms, te_ms = t.tolist()
    if rank != 0:
        return None
    apply_ms = sum(s.apply_ms for s in stats) / max(1, sum(s.apply_timed for s in stats))
    flops = FLOPS_PER_CELL_P2 * C
    achieved = flops / (apply_ms * 1e-3) / 1e12
    value = world * n * args.steps / (t_ms * 1e-3)
    line = {
        "metric": "Poisson GMG-CG solve DoF/s at 1e-8 residual",
        "value": value, "unit": "DoF/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (manufactured sin-product right-hand side, kappa = 1)",
        "config": dict(WORKLOAD, parallelism=f"replicas{world}"),
        "iterations": stats[-1].iterations, "rel_residual": stats[-1].rel_residual,
        "max_nodal_error_vs_exact": nodal_err, "setup_s": setup_s,
        "e2e": {"value": world * n * args.steps / (te_ms * 1e-3), "unit": "DoF/s",
                "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n},
        "gpu_launches": int(launches),
        "roofline": {"kernel": "k_apply<2,double> (FP64 P2 matrix-free operator)", "bound": "alu",
                     "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                     "apply_ms": apply_ms, "flops_per_launch": flops,
                     "peak_source": "nominal GB300 FP64 (recipe table); no measured FP64 peak in MEASURED_PEAKS.json"},
        "clocks": clk,
    }
    return line


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        r = run_oracle(args.warmup + args.steps)
        times = r["times"][args.warmup:]
        value = r["n"] * len(times) / sum(times)
        cb = {"value": value, "unit": "DoF/s", "cores": 1, "kind": "oracle", "sample": sample_desc(r)}
        print(json.dumps({"impl": "reference", "metric": "Poisson GMG-CG solve DoF/s at 1e-8 residual",
                          "value": value, "unit": "DoF/s", "n_gpus": args.gpus, "steps": args.steps,
                          "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": dict(WORKLOAD, parallelism="cpu"),
                          "cpu_baseline": cb,
                          "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world, local_rank)
    if rank == 0 and line is not None:
        if world == 1 and not args.no_cpu_baseline:
            r = run_oracle(1)
            line["cpu_baseline"] = {"value": r["n"] / r["times"][0], "unit": "DoF/s", "cores": 1, "kind": "oracle",
                                    "sample": sample_desc(r)}
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
