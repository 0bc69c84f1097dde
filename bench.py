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

--impl reference times the CPU FP64 oracle (assembled CSR + GMG-PCG, the CSR
products split over the host's cores) on the same workload, since the paper
ships no runnable code.

--case OP runs one kernel case a few times inside the NVTX range "case" (for
profilers: ``ncu --nvtx --nvtx-include case/``) and prints its mean time.

Multi-GPU (torchrun, N>1): the solve does not shard; every rank
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
F64_MODE = 1  # FE_F64_DOUBLE_FLOAT: the library default for FP64 operator applications
# Algorithmic bytes per dof of one matrix-free application (each array counted once; P2, kappa = 1):
# x read + y write (8 + 8 in FP64, 4 + 4 in FP32), tet->dof map (0.75 tets/dof x 10 x 4 B = 30 B),
# vertex coordinates (1/8 vertex per dof x 24 B = 3 B).
BYTES_PER_DOF_P2 = {"f64": 49.0, "f32": 41.0}
# DRAM bytes per launch of the FP64 operator kernel on this workload (dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture of the finest level's applications inside a V-cycle of the
# P2 64^3 hierarchy, the kernel the CG iterations run; mean of 2 launches), keyed by FP64 mode; None where
# the kernel changed after the last capture.
TRAFFIC = {0: None, 1: 116.4e6, 2: None}
# Arithmetic of one P2 element application (c, d, S, four G-products, transpose),
# per tet: 151 flops in the FP64 formula with a general G (an FMA counts 2).  With
# the geometric matrix shared by every Kuhn tet (G = c M) the element matrix is
# c times one integer matrix K (82 nonzeros), applied by fixed-point limbs to
# the two tets that share a face as one unit (14 dofs, 136 nonzero integers):
# per pair 674 FP32 operations (an add, mul or FMA counts 1) = 14 products c x
# as float pairs x 4, their cut into three limbs x 8 additions, 136 x 3 FMAs,
# and per row one TwoSum (6) and one addition; 337 per tet.
FLOPS_PER_CELL_P2_F64 = 151
OPS_PER_CELL_P2_DF = 337
# Operations of one P3 element application through the gradient at the P2 nodes (fe_p3.cuh; an FMA counts 1):
# 206 additions, 165 multiplications, 284 FMAs, 22 negations (counted by tests/test_p3_element_host.py)
OPS_PER_CELL_P3 = 677
FP64_PEAK_TFLOPS = 1.25  # GB300 nominal FP64: 152 SMs x 2 FMA/clk/SM x 2 flops x 2.07 GHz (recipe table)
FP32_PEAK_TOPS = 40.3  # 152 SMs x 128 FP32 lanes x 1 operation/clk x 2.07 GHz (recipe unit counts and clock)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip the matvec/mixed/adjoint/batched side measurements")
    p.add_argument("--host-loop", action="store_true",
                   help="drive the CG iterations from the host in the timed solves (same kernels; for profilers "
                        "that do not follow launches inside conditional graph nodes)")
    c = p.add_argument_group("single-kernel case (--case): no JSON line, one timing line")
    c.add_argument("--case", choices=["apply", "vcycle", "mass", "fmg"], default=None,
                   help="fmg: one full-multigrid solve of the sin-product problem (the paper's outer solver)")
    c.add_argument("--cycles", type=int, default=1, help="V-cycles per level of --case fmg")
    c.add_argument("--degree", type=int, default=2)
    c.add_argument("--N", type=int, default=64)
    c.add_argument("--nrefine", type=int, default=0)
    c.add_argument("--dtype", choices=["f64", "f32", "bf16"], default="f64")
    c.add_argument("--reps", type=int, default=3)
    c.add_argument("--f64-mode", type=int, default=None,
                   help="0 native, 1 float pairs (best layout), 2 per tet, 3 per cube, 4 two tets per thread (P2)")
    c.add_argument("--smoother", choices=["jacobi", "patch"], default="jacobi",
                   help="preconditioner of the Chebyshev smoother (--case vcycle)")
    return p.parse_args()


def max_over_ranks(values, device=None):
    """Element-wise max of a list of floats over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_throughput(units_per_rank, steps, world, total_ms):
    """Whole-job rate: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank * steps / (total_ms * 1e-3)


PHASES = ("apply", "smooth", "transfer", "coarse", "blas1")


def phase_summary(st):
    """Per-phase, per-level device time of one profiled solve (ms), from fe_solve_stats."""
    nl = max(1, st.levels_timed)
    out = {}
    for p, name in enumerate(PHASES):
        per_level = [st.phase_ms[p][l] for l in range(nl)]
        out[name] = {"total": sum(per_level), "per_level_coarse_to_fine": per_level}
    return out


def hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def apply_bytes_per_launch(n, C, nd, val_bytes, geo_bytes, cube_map=False):
    """Algorithmic bytes of one matrix-free application: x read, y zero-fill and write,
    the dof map (int32: nd per tet, or (k+1)^3 per cube for the cube-aggregated kernel),
    per-tet geometric factors (6 values)."""
    map_bytes = (C // 6) * (27 if nd == 10 else 8) * 4 if cube_map else C * nd * 4
    return n * 3 * val_bytes + map_bytes + C * 6 * geo_bytes


def time_launches(fn, stream, reps, flush):
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for e0, e1 in ev:
        flush.zero_()
        e0.record(stream)
        fn()
        e1.record(stream)
    torch.cuda.synchronize()
    ms = sorted(a.elapsed_time(b) for a, b in ev)
    return ms[len(ms) // 2]


def quadrature_rhs_rate(fe, I, hh, nd, dev, stream, flush):
    """fe_load_vector_quadrature on the finest level of ``hh`` (f given at the 27 points of every tet, b assembled
    by the one-thread-per-tet kernel): time per call and its algorithmic bytes (f values, map, |det J|, b zero-fill
    and write) against the measured HBM bandwidth."""
    import torch
    C, n = hh.n_cells(), hh.n_dofs()
    P = hh.quadrature_points()
    fq = torch.from_numpy(I.sin_product_rhs(P.reshape(-1, 3)).reshape(C, -1)).to(dev)
    del P
    b = torch.empty(n, dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(3):
            hh.load_vector_quadrature(fq, b, stream=stream)
        ms = time_launches(lambda: hh.load_vector_quadrature(fq, b, stream=stream), stream, 10, flush)
    byt = C * (fe.FE_QUAD_POINTS * 8 + nd * 4 + 8) + 2 * 8 * n
    peak, src = hbm_peak()
    return {"ms": ms, "cells": C, "dofs": n, "algorithmic_bytes": byt, "GB_per_s": byt / (ms * 1e-3) / 1e9,
            "hbm_frac": byt / (ms * 1e-3) / 1e9 / peak, "hbm_peak_source": src}


def extras(fe, I, h, dev, stream, flush):
    """Side measurements: matvec rates, mixed precision (128^3), adjoint (96^3 P1), batched (64 problems)."""
    import numpy as np
    import torch
    out = {}
    peak, src = hbm_peak()
    # ---- matvec on the benchmark's fine level (P2 64^3)
    n, C = h.n_dofs(), h.n_cells()
    mv = {}
    for name, dt, tdt, vb, gb, cube in (("f64", fe.FE_F64, torch.float64, 8, 8, False),
                                         ("f32", fe.FE_F32, torch.float32, 4, 4, True),
                                         ("bf16_tensor_core", fe.FE_BF16, torch.float32, 4, 4, False)):
        x = torch.rand(n, dtype=tdt, device=dev)
        y = torch.empty_like(x)
        with torch.cuda.stream(stream):
            for _ in range(3):
                h.apply_operator(x, y, dtype=dt, stream=stream)
            ms = time_launches(lambda: h.apply_operator(x, y, dtype=dt, stream=stream), stream, 10, flush)
        byt = apply_bytes_per_launch(n, C, 10, vb, gb, cube)
        sb = BYTES_PER_DOF_P2["f64" if vb == 8 else "f32"] * n
        mv[name] = {"ms": ms, "GDoF_per_s": n / (ms * 1e-3) / 1e9,
                    "hbm_frac_survey_bytes": sb / (ms * 1e-3) / 1e9 / peak,
                    "GB_per_s_kernel_bytes": byt / (ms * 1e-3) / 1e9,
                    "hbm_frac_kernel_bytes": byt / (ms * 1e-3) / 1e9 / peak, "kernel_bytes_per_dof": byt / n}
    out["matvec_p2_64cubed"] = dict(mv, hbm_peak_gbs=peak, hbm_peak_source=src)
    # ---- the load vector by quadrature (f at the 27 points of every tet) on the same level
    try:
        out["quadrature_load_vector_p2_64cubed"] = quadrature_rhs_rate(fe, I, h, 10, dev, stream, flush)
    except Exception as exc:  # a side measurement never stops the others
        out["quadrature_load_vector_p2_64cubed"] = {"error": repr(exc)[:300]}
    # ---- the benchmark solve with the native FP64 operator, for comparison
    u_n = torch.empty(n, dtype=torch.float64, device=dev)
    f_n = torch.from_numpy(I.sin_product_rhs(h.dof_coordinates())).to(dev)
    h.set_f64_mode(fe.FE_F64_NATIVE)
    with torch.cuda.stream(stream):
        h.solve(f_n, u_n, rtol=1e-8, stream=stream)
        ms = time_launches(lambda: h.solve(f_n, u_n, rtol=1e-8, stream=stream), stream, 3, flush)
        st = h.solve(f_n, u_n, rtol=1e-8, stream=stream)
    h.set_f64_mode(F64_MODE)
    out["native_fp64_operator_solve"] = {"ms": ms, "DoF_per_s": n / (ms * 1e-3), "iterations": st.iterations,
                                         "rel_residual": st.rel_residual}
    # ---- the benchmark solve with the Chebyshev update fused into the operator launch (per-dof countdowns)
    h.set_smoother_fusion(True)
    with torch.cuda.stream(stream):
        h.solve(f_n, u_n, rtol=1e-8, stream=stream)
        ms = time_launches(lambda: h.solve(f_n, u_n, rtol=1e-8, stream=stream), stream, 3, flush)
        st = h.solve(f_n, u_n, rtol=1e-8, stream=stream)
    h.set_smoother_fusion(False)
    out["fused_smoother_solve"] = {"ms": ms, "DoF_per_s": n / (ms * 1e-3), "iterations": st.iterations,
                                   "rel_residual": st.rel_residual}
    # ---- the paper's level smoother: Chebyshev preconditioned by vertex-star patches, CG and full multigrid
    ue = torch.from_numpy(I.sin_product(h.dof_coordinates()))
    h.set_smoother(fe.FE_SMOOTHER_PATCH)
    pt = {"what": "Chebyshev(2) preconditioned by vertex-star patches (additive, exact 15x15 local solves)",
          "lambda_max": [h.lambda_max(l) for l in range(h.nlev)]}
    with torch.cuda.stream(stream):
        h.solve(f_n, u_n, rtol=1e-8, stream=stream)
        ms = time_launches(lambda: h.solve(f_n, u_n, rtol=1e-8, stream=stream), stream, 3, flush)
        st = h.solve(f_n, u_n, rtol=1e-8, stream=stream)
        pt["gmg_pcg"] = {"ms": ms, "DoF_per_s": n / (ms * 1e-3), "iterations": st.iterations,
                         "rel_residual": st.rel_residual}
        h.solve(f_n, u_n, precond=fe.FE_PC_FMG, max_it=1, stream=stream)
        ms = time_launches(lambda: h.solve(f_n, u_n, precond=fe.FE_PC_FMG, max_it=1, stream=stream), stream, 3, flush)
        st = h.solve(f_n, u_n, precond=fe.FE_PC_FMG, max_it=1, stream=stream)
        pt["full_multigrid_1_cycle"] = {"ms": ms, "rel_residual": st.rel_residual,
                                        "max_nodal_error_vs_exact": float((u_n.cpu() - ue).abs().max())}
    h.set_smoother(fe.FE_SMOOTHER_JACOBI)
    out["patch_smoother_p2_64cubed"] = pt
    # ---- full multigrid as the whole solve (the paper's outer solver) on the same problem
    fm = {"what": "one full-multigrid cycle (restrict b to all levels, coarse Cholesky, per finer level: "
                  "interpolate, V-cycles), P2 64^3, 4 levels",
          "cg_max_nodal_error_vs_exact": float((u_n.cpu() - ue).abs().max())}
    for cyc in (1, 2):
        with torch.cuda.stream(stream):
            h.solve(f_n, u_n, precond=fe.FE_PC_FMG, max_it=cyc, stream=stream)
            ms = time_launches(lambda: h.solve(f_n, u_n, precond=fe.FE_PC_FMG, max_it=cyc, stream=stream), stream, 5,
                               flush)
            st = h.solve(f_n, u_n, precond=fe.FE_PC_FMG, max_it=cyc, stream=stream)
        fm[f"vcycles_per_level_{cyc}"] = {"ms": ms, "DoF_per_s": n / (ms * 1e-3), "rel_residual": st.rel_residual,
                                          "max_nodal_error_vs_exact": float((u_n.cpu() - ue).abs().max())}
    out["fmg_p2_64cubed"] = fm
    # ---- mixed precision on P2 128^3 (5 levels): time to the same 1e-8 FP64 residual
    h2 = fe.Hierarchy(8, 4, 2)
    f2 = torch.from_numpy(I.sin_product_rhs(h2.dof_coordinates())).to(dev)
    ref = torch.empty(h2.n_dofs(), dtype=torch.float64, device=dev)
    u2 = torch.empty_like(ref)
    mp = {"workload": "P2 UnitCubeMesh 128^3, 5 levels, rtol 1e-8", "dofs": h2.n_dofs()}
    # FP32 matvec on the 128^3 level (inputs 8x larger than L2)
    n2 = h2.n_dofs()
    x32 = torch.rand(n2, dtype=torch.float32, device=dev)
    y32 = torch.empty_like(x32)
    with torch.cuda.stream(stream):
        for _ in range(3):
            h2.apply_operator(x32, y32, dtype=fe.FE_F32, stream=stream)
        ms = time_launches(lambda: h2.apply_operator(x32, y32, dtype=fe.FE_F32, stream=stream), stream, 10, flush)
    byt = apply_bytes_per_launch(n2, h2.n_cells(), 10, 4, 4, cube_map=True)
    sb = BYTES_PER_DOF_P2["f32"] * n2
    out["matvec_p2_128cubed_f32"] = {"ms": ms, "GDoF_per_s": n2 / (ms * 1e-3) / 1e9,
                                     "hbm_frac_survey_bytes": sb / (ms * 1e-3) / 1e9 / peak,
                                     "survey_bytes_per_dof": BYTES_PER_DOF_P2["f32"],
                                     "kernel_bytes_per_dof": byt / n2, "GB_per_s_kernel_bytes": byt / (ms * 1e-3) / 1e9,
                                     "hbm_frac_kernel_bytes": byt / (ms * 1e-3) / 1e9 / peak,
                                     "kernel_bytes_model": "x 4 + y zero-fill and write 8 + cube->dof map 27 x 4 per "
                                                           "cube + per-tet geometric factors 6 x 4 per tet",
                                     "hbm_peak_gbs": peak, "hbm_peak_source": src}
    del x32, y32
    for name, prec in (("f64", fe.FE_PREC_F64), ("mixed_f32", fe.FE_PREC_MIXED_F32),
                       ("mixed_bf16_tensor_core", fe.FE_PREC_MIXED_BF16)):
        target = ref if prec == fe.FE_PREC_F64 else u2
        try:
            with torch.cuda.stream(stream):
                h2.solve(f2, target, rtol=1e-8, precision=prec, max_it=30, stream=stream)
                ms = time_launches(lambda: h2.solve(f2, target, rtol=1e-8, precision=prec, max_it=30, stream=stream),
                                   stream, 3, flush)
                st = h2.solve(f2, target, rtol=1e-8, precision=prec, max_it=30, stream=stream)
        except fe.FeError as exc:
            mp[name] = {"error": str(exc)}
            continue
        e = {"ms": ms, "DoF_per_s": h2.n_dofs() / (ms * 1e-3), "iterations": st.iterations,
             "outer": st.outer_iterations, "rel_residual": st.rel_residual, "fp64_applies": st.fine_applies_f64}
        if prec != fe.FE_PREC_F64:
            e["rel_l2_diff_vs_fp64_gpu_solution"] = float(torch.linalg.norm(u2 - ref) / torch.linalg.norm(ref))
        e["max_nodal_error_vs_exact"] = float((target.cpu() - torch.from_numpy(
            I.sin_product(h2.dof_coordinates()))).abs().max())
        mp[name] = e
    if "ms" in mp.get("f64", {}) and "ms" in mp.get("mixed_f32", {}):
        mp["speedup_mixed_f32_vs_f64"] = mp["f64"]["ms"] / mp["mixed_f32"]["ms"]
    out["mixed_precision_p2_128cubed"] = mp
    h2.close()
    del f2, ref, u2
    # ---- adjoint gradient on P1 96^3 with a GRF kappa (forward + adjoint solve + gradient kernel)
    h3 = fe.Hierarchy(12, 3, 1)
    kap = torch.from_numpy(I.grf_kappa(h3.cell_centroids(), device=dev)).to(dev)
    h3.set_coefficient(kap)
    X3 = h3.dof_coordinates()
    f3 = torch.ones(h3.n_dofs(), dtype=torch.float64, device=dev)
    ud = torch.from_numpy(I.target_field(X3)).to(dev)
    g = torch.empty(h3.n_cells(), dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        h3.adjoint_gradient(f3, ud, g, rtol=1e-8, stream=stream)
        ms = time_launches(lambda: h3.adjoint_gradient(f3, ud, g, rtol=1e-8, stream=stream), stream, 3, flush)
    out["adjoint_p1_96cubed"] = {"ms": ms, "cells": h3.n_cells(), "dofs": h3.n_dofs(),
                                 "what": "forward GMG-PCG + adjoint GMG-PCG + per-cell gradient kernel, rtol 1e-8"}
    h3.close()
    # ---- batched: 64 problems, one persistent launch
    table = I.batched_problem_table()
    B = fe.Batch([(N // 8, 3, k) for N, k in table])
    fs, us = [], []
    for p, hp in enumerate(B.problems):
        hp.set_coefficient(torch.from_numpy(I.grf_kappa(hp.cell_centroids(), seed=100 + p, device=dev)).to(dev))
        fs.append(torch.ones(hp.n_dofs(), dtype=torch.float64, device=dev))
        us.append(torch.empty(hp.n_dofs(), dtype=torch.float64, device=dev))
    with torch.cuda.stream(stream):
        B.solve(fs, us, rtol=1e-8, stream=stream)  # first graph solve autotunes
        ms = time_launches(lambda: B.solve(fs, us, rtol=1e-8, stream=stream), stream, 3, flush)
        st = B.solve(fs, us, rtol=1e-8, stream=stream)
    tot = sum(hp.n_dofs() for hp in B.problems)
    out["batched_64"] = {"ms": ms, "total_dofs": tot, "DoF_per_s": tot / (ms * 1e-3),
                         "max_iterations": max(s.iterations for s in st),
                         "max_rel_residual": max(s.rel_residual for s in st), "schedule": B.schedule()}
    with torch.cuda.stream(stream):  # the persistent launch's wall time by phase and level (direct launch)
        stp = B.solve(fs, us, rtol=1e-8, profile=1, stream=stream)
    out["batched_64"]["phases_ms_profiled"] = phase_summary(stp[0])
    out["batched_64"]["profiled_solve_ms"] = stp[0].solve_ms
    # the same 64 problems solved one after another with the single-problem solver (for comparison)
    with torch.cuda.stream(stream):
        for hp, fp, up in zip(B.problems, fs, us):
            hp.solve(fp, up, rhs_kind=fe.FE_RHS_NODAL_F, rtol=1e-8, stream=stream)
        ms_seq = time_launches(lambda: [hp.solve(fp, up, rtol=1e-8, stream=stream)
                                        for hp, fp, up in zip(B.problems, fs, us)], stream, 3, flush)
    out["batched_64"]["sequential_single_solves_ms"] = ms_seq
    B.close()
    # ---- P3 (the paper's degree) on UnitCubeMesh 32^3, 4 levels: operator rates and solves
    h4 = fe.Hierarchy(4, 3, 3)
    n4, C4 = h4.n_dofs(), h4.n_cells()
    p3 = {"workload": "P3 UnitCubeMesh 32^3, 4 levels (coarse 4^3), rtol 1e-8", "dofs": n4, "cells": C4}
    ops_per_cell = OPS_PER_CELL_P3  # the element through the gradient at the P2 nodes (fe_p3.cuh)
    for name, dtp, tdt, mode in (("apply_f64", fe.FE_F64, torch.float64, F64_MODE),
                                 ("apply_f64_native", fe.FE_F64, torch.float64, fe.FE_F64_NATIVE),
                                 ("apply_f32", fe.FE_F32, torch.float32, F64_MODE)):
        h4.set_f64_mode(mode)
        x4 = torch.rand(n4, dtype=tdt, device=dev)
        y4 = torch.empty_like(x4)
        with torch.cuda.stream(stream):
            for _ in range(3):
                h4.apply_operator(x4, y4, dtype=dtp, stream=stream)
            ms = time_launches(lambda: h4.apply_operator(x4, y4, dtype=dtp, stream=stream), stream, 10, flush)
        # the element's operations per tet per second (in float pairs: FP64-equivalent operations)
        tops = ops_per_cell * C4 / (ms * 1e-3) / 1e12
        p3[name] = {"ms": ms, "GDoF_per_s": n4 / (ms * 1e-3) / 1e9, "element_T_ops_per_s": tops}
    h4.set_f64_mode(F64_MODE)
    try:
        p3["quadrature_load_vector"] = quadrature_rhs_rate(fe, I, h4, 20, dev, stream, flush)
    except Exception as exc:
        p3["quadrature_load_vector"] = {"error": repr(exc)[:300]}
    p3["element_ops_per_tet"] = ops_per_cell
    p3["apply_f64"]["arithmetic"] = "float pairs on the FP32 pipes (k_apply_df3)"
    p3["apply_f64_native"]["arithmetic"] = "FP64 (k_apply<3, double>)"
    # FP64 issue rate in operations: half the nominal flop rate (an FMA is 2 flops)
    p3["apply_f64_native"]["frac_of_nominal_fp64_rate"] = p3["apply_f64_native"]["element_T_ops_per_s"] / (
        FP64_PEAK_TFLOPS / 2)
    p3["apply_f32"]["frac_of_fp32_issue_rate"] = p3["apply_f32"]["element_T_ops_per_s"] / FP32_PEAK_TOPS
    f4 = torch.from_numpy(I.sin_product_rhs(h4.dof_coordinates())).to(dev)
    u4 = torch.empty_like(f4)
    for name, prec in (("solve_f64", fe.FE_PREC_F64), ("solve_mixed_f32", fe.FE_PREC_MIXED_F32),
                       ("solve_mixed_bf16_tensor_core", fe.FE_PREC_MIXED_BF16)):
        with torch.cuda.stream(stream):
            h4.solve(f4, u4, rtol=1e-8, precision=prec, stream=stream)
            ms = time_launches(lambda: h4.solve(f4, u4, rtol=1e-8, precision=prec, stream=stream), stream, 3, flush)
            st = h4.solve(f4, u4, rtol=1e-8, precision=prec, stream=stream)
        p3[name] = {"ms": ms, "DoF_per_s": n4 / (ms * 1e-3), "iterations": st.iterations,
                    "outer": st.outer_iterations, "rel_residual": st.rel_residual,
                    "max_nodal_error_vs_exact": float((u4.cpu() - torch.from_numpy(
                        I.sin_product(h4.dof_coordinates()))).abs().max())}
    # the paper's solver on P3: full multigrid (1 or 2 V-cycles per level) smoothed by Chebyshev(2) with
    # vertex-star patches, direct coarse solve; error against the exact solution vs. the discretisation error
    ue4 = torch.from_numpy(I.sin_product(h4.dof_coordinates()))
    fmg = {}
    for sm_name, sm in (("jacobi", fe.FE_SMOOTHER_JACOBI), ("patch", fe.FE_SMOOTHER_PATCH)):
        h4.set_smoother(sm)
        for cyc in (1, 2):
            with torch.cuda.stream(stream):
                h4.solve(f4, u4, precond=fe.FE_PC_FMG, max_it=cyc, stream=stream)
                ms = time_launches(lambda: h4.solve(f4, u4, precond=fe.FE_PC_FMG, max_it=cyc, stream=stream),
                                   stream, 3, flush)
                st = h4.solve(f4, u4, precond=fe.FE_PC_FMG, max_it=cyc, stream=stream)
            fmg[f"{sm_name}_{cyc}_cycles"] = {"ms": ms, "rel_residual": st.rel_residual,
                                              "max_nodal_error_vs_exact": float((u4.cpu() - ue4).abs().max())}
        with torch.cuda.stream(stream):
            h4.solve(f4, u4, rtol=1e-8, stream=stream)
            ms = time_launches(lambda: h4.solve(f4, u4, rtol=1e-8, stream=stream), stream, 3, flush)
            st = h4.solve(f4, u4, rtol=1e-8, stream=stream)
        fmg[f"{sm_name}_gmg_pcg_1e-8"] = {"ms": ms, "iterations": st.iterations,
                                         "max_nodal_error_vs_exact": float((u4.cpu() - ue4).abs().max())}
    h4.set_smoother(fe.FE_SMOOTHER_JACOBI)
    p3["paper_solver"] = dict(fmg, what="full multigrid (the paper's outer solver) and GMG-PCG, each with Jacobi "
                                         "or vertex-star patch (the paper's PatchPC) Chebyshev(2) smoothing")
    out["p3_32cubed"] = p3
    h4.close()
    # ---- the paper's Poisson problem at full size: P3 on UnitCubeMesh 128^3 (57,066,625 dofs), 5 levels from 8^3
    t0 = time.perf_counter()
    h5 = fe.Hierarchy(8, 4, 3)
    pw = {"workload": "P3 UnitCubeMesh 128^3 (the paper's Poisson problem), 5 levels from 8^3, f = 3 pi^2 sin sin sin",
          "dofs": h5.n_dofs(), "cells": h5.n_cells(), "setup_s": time.perf_counter() - t0}
    X5 = h5.dof_coordinates()
    f5 = torch.from_numpy(I.sin_product_rhs(X5)).to(dev)
    ue5 = torch.from_numpy(I.sin_product(X5)).to(dev)
    del X5
    u5 = torch.empty_like(f5)

    def run5(name, reps=2, **kw):
        with torch.cuda.stream(stream):
            st = h5.solve(f5, u5, stream=stream, **kw)
            ms = time_launches(lambda: h5.solve(f5, u5, stream=stream, **kw), stream, reps, flush)
        pw[name] = {"ms": ms, "DoF_per_s": h5.n_dofs() / (ms * 1e-3), "iterations": st.iterations,
                    "max_nodal_error_vs_exact": float((u5 - ue5).abs().max())}

    run5("jacobi_gmg_pcg_1e-8", rtol=1e-8)
    run5("mixed_f32_gmg_pcg_1e-8", rtol=1e-8, precision=fe.FE_PREC_MIXED_F32)
    run5("jacobi_full_multigrid_2_cycles", precond=fe.FE_PC_FMG, max_it=2)
    t0 = time.perf_counter()
    h5.set_smoother(fe.FE_SMOOTHER_PATCH)
    torch.cuda.synchronize()
    pw["patch_setup_s"] = time.perf_counter() - t0
    run5("paper_solver_full_multigrid_patch_1_cycle", precond=fe.FE_PC_FMG, max_it=1)
    run5("paper_solver_full_multigrid_patch_2_cycles", precond=fe.FE_PC_FMG, max_it=2)
    out["paper_poisson_p3_128cubed"] = pw
    h5.close()
    del f5, ue5, u5
    # ---- the paper's own hierarchy for that problem: 4 levels from UnitCubeMesh 16^3 (103,823 interior coarse
    # unknowns), the coarse level solved directly with the blocked band Cholesky factor
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    t0 = time.perf_counter()
    h6 = fe.Hierarchy(16, 3, 3)
    torch.cuda.synchronize()
    ph = {"workload": "P3 UnitCubeMesh 128^3 as the paper's 4-level hierarchy from 16^3, direct coarse solve "
                      "(blocked band Cholesky)", "dofs": h6.n_dofs(), "setup_s": time.perf_counter() - t0,
          "coarse": h6.coarse_info(), "device_bytes_after_setup": free0 - torch.cuda.mem_get_info()[0]}
    X6 = h6.dof_coordinates()
    f6 = torch.from_numpy(I.sin_product_rhs(X6)).to(dev)
    ue6 = torch.from_numpy(I.sin_product(X6)).to(dev)
    del X6
    u6 = torch.empty_like(f6)

    def run6(name, reps=2, **kw):
        with torch.cuda.stream(stream):
            st = h6.solve(f6, u6, stream=stream, **kw)
            ms = time_launches(lambda: h6.solve(f6, u6, stream=stream, **kw), stream, reps, flush)
            stp = h6.solve(f6, u6, stream=stream, profile=1, **kw)
        ph[name] = {"ms": ms, "DoF_per_s": h6.n_dofs() / (ms * 1e-3), "iterations": st.iterations,
                    "max_nodal_error_vs_exact": float((u6 - ue6).abs().max()),
                    "coarse_solve_ms_profiled": stp.phase_ms[fe.FE_PHASE_COARSE][0],
                    "phases_ms_profiled": phase_summary(stp)}

    run6("jacobi_gmg_pcg_1e-8", rtol=1e-8)
    run6("jacobi_full_multigrid_2_cycles", precond=fe.FE_PC_FMG, max_it=2)
    t0 = time.perf_counter()
    h6.set_smoother(fe.FE_SMOOTHER_PATCH)
    torch.cuda.synchronize()
    ph["patch_setup_s"] = time.perf_counter() - t0
    run6("paper_solver_full_multigrid_patch_1_cycle", precond=fe.FE_PC_FMG, max_it=1)
    run6("paper_solver_full_multigrid_patch_2_cycles", precond=fe.FE_PC_FMG, max_it=2)
    ph["device_bytes_with_patches"] = free0 - torch.cuda.mem_get_info()[0]
    out["paper_poisson_p3_128cubed_paper_hierarchy"] = ph
    h6.close()
    del f6, ue6, u6
    return out


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
# The oracle runs in its own interpreter (started before this process touches
# the GPU): it builds the benchmark's hierarchy (assembled CSR on every level,
# prolongations, Lanczos estimates, coarse Cholesky), then waits for one line
# on stdin before its timed solves, so that its set-up overlaps the GPU run
# and its solves do not share the host with it.
ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import build_oracle
build_oracle.build()
from oracle import fe_oracle as O
import fe_inputs as I
N0, nref, k, steps = {N0}, {nref}, {k}, {steps}
cores = O.THREADS
t0 = time.time()
h = O.Hierarchy(N0, nref, k)
L = h.fine
b = O.load_vector(L, I.sin_product_rhs(L.space.coords))
setup = time.time() - t0
print(json.dumps({{"ready": True, "setup_s": setup}}), flush=True)
sys.stdin.readline()
times, its = [], []
for s in range(steps):
    t = time.time()
    u, it, hist = O.solve(h, b, rtol=1e-8)
    times.append(time.time() - t)
    its.append(it)
rel_res = hist[-1]
err = float(np.abs(u - I.sin_product(L.space.coords)).max())
# one more solve with the CSR products on a single thread
O.THREADS = 1
t = time.time()
O.solve(h, b, rtol=1e-8)
t1 = time.time() - t
O.THREADS = cores
# the assembled fine-level CSR product alone (the oracle's operator application)
x = I.random_vector(L.n, 1)
spmv = {{}}
for th in (cores, 1):
    O.matvec(L.A, x, threads=th)
    t = time.time()
    for _ in range(10):
        O.matvec(L.A, x, threads=th)
    spmv[th] = (time.time() - t) / 10
print(json.dumps({{"n": int(L.n), "setup_s": setup, "times": times, "iterations": its, "rel_res": rel_res,
                  "max_nodal_error_vs_exact": err, "time_1thread": t1, "spmv_s": spmv[cores],
                  "spmv_1thread_s": spmv[1], "nnz": int(L.A.nnz), "cores": cores,
                  "threaded_products": O._csr_lib() is not None}}))
"""


class OracleRun:
    """The oracle on the benchmark's own workload in a subprocess; ``start`` before any GPU work."""

    def __init__(self, steps):
        env = dict(os.environ)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env.pop(k, None)
        code = ORACLE_SNIPPET.format(root=ROOT, N0=WORKLOAD["coarse_mesh"], nref=WORKLOAD["levels"] - 1,
                                     k=WORKLOAD["degree"], steps=steps)
        self.proc = subprocess.Popen([sys.executable, "-c", code], stdin=subprocess.PIPE, stdout=subprocess.PIPE,
                                     stderr=subprocess.PIPE, text=True, env=env)

    def result(self, timeout=1800):
        """Wait for the set-up, release the timed solves and return their record."""
        p = self.proc
        try:
            line = p.stdout.readline()
            if not line:
                raise RuntimeError(p.stderr.read()[-2000:])
            p.stdin.write("go\n")
            p.stdin.flush()
            out, err = p.communicate(timeout=timeout)
        except Exception:
            p.kill()
            raise
        if p.returncode != 0:
            raise RuntimeError(err[-2000:])
        return json.loads(out.strip().splitlines()[-1])


def oracle_details(r):
    """Set-up time, iterations, 1-thread solve and the CSR operator product rates of the oracle run."""
    return {"setup_s": r["setup_s"], "iterations": r["iterations"][-1], "rel_residual": r["rel_res"],
            "max_nodal_error_vs_exact": r["max_nodal_error_vs_exact"],
            "value_1thread": r["n"] / r["time_1thread"], "cores_1thread": 1,
            "csr_spmv_dof_per_s": r["n"] / r["spmv_s"], "csr_spmv_dof_per_s_1thread": r["n"] / r["spmv_1thread_s"],
            "csr_nnz": r["nnz"], "host_cores_in_affinity": r["cores"]}


def sample_desc(r):
    thr = (f"CSR products on {r['cores']} OpenMP threads (the rest numpy/scipy, one thread)"
           if r["threaded_products"] else "scipy CSR products on one thread")
    return (f"oracle GMG-PCG solve of the benchmark workload itself (P2 UnitCubeMesh 64^3, {r['n']} dofs, 4 levels, "
            f"assembled CSR), rtol 1e-8, {len(r['times'])} timed solve(s), set-up {r['setup_s']:.0f} s excluded; "
            f"{thr}")


# --------------------------------------------------------------- case
def run_case(a):
    """One kernel case a few times on a single mesh (or hierarchy) inside the NVTX range "case"."""
    import numpy as np
    import torch

    from paper_2104_08012_gb300 import build as _build
    _build.build()
    import paper_2104_08012_gb300 as fe
    dt = {"f64": fe.FE_F64, "f32": fe.FE_F32, "bf16": fe.FE_BF16}[a.dtype]
    tdt = torch.float64 if a.dtype == "f64" else torch.float32
    N0 = a.N >> a.nrefine
    h = fe.Hierarchy(N0, a.nrefine, a.degree)
    if a.f64_mode is not None:
        h.set_f64_mode(a.f64_mode)
    if a.smoother == "patch":
        h.set_smoother(fe.FE_SMOOTHER_PATCH)
    n = h.n_dofs()
    if a.case == "fmg":
        import fe_inputs as I
        x = torch.from_numpy(I.sin_product_rhs(h.dof_coordinates())).to("cuda", torch.float64)
        h.solve(x, torch.empty_like(x), precond=fe.FE_PC_FMG, max_it=a.cycles)  # build the graph outside the range
    else:
        x = torch.from_numpy(np.random.default_rng(0).uniform(-1, 1, n)).to("cuda", tdt)
    y = torch.empty_like(x)
    s = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.reps)]
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("case")
    for e0, e1 in evs:
        e0.record(s)
        if a.case == "apply":
            h.apply_operator(x, y, dtype=dt, stream=s)
        elif a.case == "mass":
            h.apply_mass(x, y, stream=s)
        elif a.case == "fmg":
            h.solve(x, y, precond=fe.FE_PC_FMG, max_it=a.cycles, stream=s)
        else:
            h.vcycle(x, y, dtype=dt, stream=s)
        e1.record(s)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    print(f"{a.case} P{a.degree} N={a.N} {a.dtype}: n={n} cells={h.n_cells()} ms/launch={np.mean(ms):.4f} "
          f"(min {np.min(ms):.4f})")
    h.close()


# --------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank, oracle=None):
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
    h.set_f64_mode(F64_MODE)
    n, C = h.n_dofs(), h.n_cells()
    assert n == WORKLOAD["dofs"] and C == WORKLOAD["cells"]
    f_host = I.sin_product_rhs(h.dof_coordinates())
    setup_s = time.time() - t_setup
    f = torch.from_numpy(f_host).to(dev)
    u = torch.empty(n, dtype=torch.float64, device=dev)
    opts_prof = fe.default_opts(rtol=WORKLOAD["rtol"], profile=1)
    opts = opts_prof if args.host_loop else fe.default_opts(rtol=WORKLOAD["rtol"])
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)

    def step(rhs, out, o=opts):
        return h.solve(rhs, out, opts=o, stream=stream)

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
    # operator-apply durations for the roofline: the same solves with CUDA events around
    # every fine-level application (host-driven CG loop), after the timed region
    pstats = []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            pstats.append(step(f, u, opts_prof))
    torch.cuda.synchronize()
    # correctness of the last solve: relative residual reported by the FP64 recurrence and an
    # independent check of the error against the analytic solution at the nodes
    u_host = u.cpu().numpy()
    nodal_err = float(np.abs(u_host - I.sin_product(h.dof_coordinates())).max())
    t_ms, te_ms = max_over_ranks([t_ms, te_ms], device=dev)
    extra = None
    if rank == 0 and not args.no_extras:
        try:
            extra = extras(fe, I, h, dev, stream, flush)
        except Exception as exc:  # side measurements never break the main line
            extra = {"error": repr(exc)[:300]}
    if rank != 0:
        return None
    apply_ms = sum(s.apply_ms for s in pstats) / max(1, sum(s.apply_timed for s in pstats))
    peak_hbm, hsrc = hbm_peak()
    # the bytes view of the scope table: algorithmic bytes per dof x dofs / event-timed launch duration
    byt = BYTES_PER_DOF_P2["f64"] * n
    achieved_gbs = byt / (apply_ms * 1e-3) / 1e9
    if F64_MODE == fe.FE_F64_DOUBLE_FLOAT:
        kname = ("k_apply_lp<KuhnPair> (FP64 operator on the FP32 pipes: exact fixed-point limbs of c x against the "
                 "integer stiffness of the two Kuhn tets that share a face, applied as one unit of 14 dofs; "
                 "persistent, map rows staged in shared memory by cp.async)")
        ops, opeak, ounit = OPS_PER_CELL_P2_DF * C, FP32_PEAK_TOPS, "T FP32 op/s"
        oderiv = ("337 FP32 operations per tet of the limb element (674 per pair) x cells / launch duration, against the "
                  "nominal FP32 issue rate 152 SMs x 128 lanes x 1 op/clk x 2.07 GHz = 40.3 T op/s (no measured FP32 "
                  "peak exists)")
    else:
        kname = "k_apply<2,double> (native FP64 operator)"
        ops, opeak, ounit = FLOPS_PER_CELL_P2_F64 * C, FP64_PEAK_TFLOPS, "TFLOP/s"
        oderiv = "151 FP64 flops per tet x cells / launch duration, against the nominal 1.25 TFLOP/s FP64 rate"
    value = job_throughput(n, args.steps, world, t_ms)
    line = {
        "metric": "Poisson GMG-CG solve DoF/s at 1e-8 residual",
        "value": value, "unit": "DoF/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 (operator on the FP32 pipes, ~47-bit)" if F64_MODE == fe.FE_F64_DOUBLE_FLOAT else "f64",
        "data": "synthetic (manufactured sin-product right-hand side, kappa = 1)",
        "config": dict(WORKLOAD, parallelism=f"replicas{world}",
                       f64_operator="P2 element as exact fixed-point limbs of float-pair products on the FP32 "
                                    "pipes (~47-bit); FP64 vectors, reductions, transfers, smoother updates, coarse "
                                    "Cholesky"
                       if F64_MODE == 1 else "native FP64"),
        "iterations": stats[-1].iterations, "rel_residual": stats[-1].rel_residual,
        "max_nodal_error_vs_exact": nodal_err, "setup_s": setup_s,
        "e2e": {"value": job_throughput(n, args.steps, world, te_ms), "unit": "DoF/s",
                "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n},
        "gpu_launches": int(launches),
        "roofline": {"kernel": kname, "bound": "hbm", "achieved": achieved_gbs, "peak": peak_hbm, "unit": "GB/s",
                     "frac": achieved_gbs / peak_hbm, "frac_hbm": achieved_gbs / peak_hbm,
                     "traffic": TRAFFIC.get(F64_MODE), "apply_ms": apply_ms,
                     "algorithmic_bytes_per_launch": byt, "bytes_per_dof": BYTES_PER_DOF_P2["f64"],
                     "bytes_model": "x read 8 + y write 8 + tet->dof map 30 + vertex coordinates 3 B per dof (P2, "
                                    "kappa = 1)",
                     "peak_source": f"{hsrc} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if hsrc == "measured"
                     else "fallback 6.8 TB/s",
                     "limiter": "instruction issue and gather latency, not DRAM (ncu: issue 65%, FP64 pipe 48%)",
                     "alu_issue_view_nominal": {"achieved": ops / (apply_ms * 1e-3) / 1e12, "peak": opeak,
                                                "unit": ounit, "frac": ops / (apply_ms * 1e-3) / 1e12 / opeak,
                                                "derivation": oderiv},
                     "apply_timing": "CUDA events around each fine-level apply of the same solves (host-driven "
                                     "CG loop), run after the timed region"},
        "clocks": clk,
    }
    if pstats and hasattr(pstats[-1], "phase_ms"):
        line["phases_ms_per_solve"] = phase_summary(pstats[-1])
    if extra is not None:
        line["extras"] = extra
    return line


def summary(line):
    """The headline figures, gathered at the end of the line."""
    ex = line.get("extras") or {}
    out = {"solve_dofs_per_s": line["value"], "e2e_dofs_per_s": line["e2e"]["value"],
           "fp64_apply_hbm_frac_survey_bytes": line["roofline"]["frac_hbm"]}
    nat = ex.get("native_fp64_operator_solve", {})
    if "DoF_per_s" in nat:
        out["native_fp64_solve_dofs_per_s"] = nat["DoF_per_s"]
    mv = ex.get("matvec_p2_128cubed_f32", {})
    if "hbm_frac_survey_bytes" in mv:
        out["matvec_f32_128_hbm_frac_survey_bytes"] = mv["hbm_frac_survey_bytes"]
    mp = ex.get("mixed_precision_p2_128cubed", {})
    for name, key in (("mixed_f32", "mixed_f32_speedup_vs_f64"), ("mixed_bf16_tensor_core", "mixed_bf16_speedup_vs_f64")):
        if "ms" in mp.get("f64", {}) and "ms" in mp.get(name, {}):
            out[key] = mp["f64"]["ms"] / mp[name]["ms"]
            out[key.replace("speedup_vs_f64", "rel_l2_vs_fp64")] = mp[name].get("rel_l2_diff_vs_fp64_gpu_solution")
    p3 = ex.get("p3_32cubed", {})
    for name, key in (("solve_mixed_f32", "p3_mixed_f32_speedup_vs_f64"),
                      ("solve_mixed_bf16_tensor_core", "p3_mixed_bf16_speedup_vs_f64")):
        if "ms" in p3.get("solve_f64", {}) and "ms" in p3.get(name, {}):
            out[key] = p3["solve_f64"]["ms"] / p3[name]["ms"]
    cb = line.get("cpu_baseline", {})
    if "value" in cb:
        out["oracle_dofs_per_s"] = cb["value"]
        out["oracle_cores"] = cb.get("cores")
        out["oracle_dofs_per_s_1thread"] = cb.get("value_1thread")
    return out


def main():
    args = parse()
    if args.case:
        run_case(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        r = OracleRun(args.warmup + args.steps).result()
        times = r["times"][args.warmup:]
        value = r["n"] * len(times) / sum(times)
        cb = {"value": value, "unit": "DoF/s", "cores": r["cores"] if r["threaded_products"] else 1,
              "kind": "oracle", "sample": sample_desc(r), **oracle_details(r)}
        print(json.dumps({"impl": "reference", "metric": "Poisson GMG-CG solve DoF/s at 1e-8 residual",
                          "value": value, "unit": "DoF/s", "n_gpus": args.gpus, "steps": args.steps,
                          "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic (manufactured sin-product right-hand side, kappa = 1)",
                          "config": dict(WORKLOAD, parallelism="cpu"), "cpu_baseline": cb,
                          "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    oracle = None
    if world == 1 and not args.no_cpu_baseline:
        oracle = OracleRun(1)  # set-up overlaps the GPU run; its solve runs afterwards
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world, local_rank)
    if rank == 0 and line is not None:
        if oracle is not None:
            try:
                r = oracle.result()
                line["cpu_baseline"] = {"value": r["n"] / r["times"][0], "unit": "DoF/s",
                                        "cores": r["cores"] if r["threaded_products"] else 1, "kind": "oracle",
                                        "sample": sample_desc(r), **oracle_details(r)}
            except Exception as exc:  # the GPU line is printed either way
                line["cpu_baseline"] = {"error": repr(exc)[:300]}
        line["summary"] = summary(line)
        print(json.dumps(line))
    elif oracle is not None:
        oracle.proc.kill()
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
