"""Run one operator kernel a few times on a single-level mesh (for profilers).

    python -m paper_2104_08012_gb300.kernel_case --op apply --degree 2 --N 64 --dtype f64 --reps 3

The launches of interest sit inside the NVTX range "case", so a profiler can
skip the setup (geometry, diagonal, eigenvalue estimate) with
``--nvtx --nvtx-include case/``.  Prints the mean CUDA-event time per launch.
"""
import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["apply", "vcycle", "mass", "fmg"], default="apply",
                    help="fmg: one full-multigrid solve of the sin-product problem (the paper's outer solver)")
    ap.add_argument("--cycles", type=int, default=1, help="V-cycles per level of --op fmg")
    ap.add_argument("--degree", type=int, default=2)
    ap.add_argument("--N", type=int, default=64)
    ap.add_argument("--nrefine", type=int, default=0)
    ap.add_argument("--dtype", choices=["f64", "f32", "bf16"], default="f64")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--f64-mode", type=int, default=None,
                    help="0 native, 1 double-float (best layout), 2 per tet, 3 per cube, 4 two tets per thread (P2)")
    ap.add_argument("--smoother", choices=["jacobi", "patch"], default="jacobi",
                    help="preconditioner of the Chebyshev smoother (--op vcycle)")
    a = ap.parse_args()
    import numpy as np
    import torch

    import paper_2104_08012_gb300 as fe
    from paper_2104_08012_gb300 import build
    build.build()
    dt = {"f64": fe.FE_F64, "f32": fe.FE_F32, "bf16": fe.FE_BF16}[a.dtype]
    tdt = torch.float64 if a.dtype == "f64" else torch.float32
    N0 = a.N >> a.nrefine
    h = fe.Hierarchy(N0, a.nrefine, a.degree)
    if a.f64_mode is not None:
        h.set_f64_mode(a.f64_mode)
    if a.smoother == "patch":
        h.set_smoother(fe.FE_SMOOTHER_PATCH)
    n = h.n_dofs()
    if a.op == "fmg":
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
        if a.op == "apply":
            h.apply_operator(x, y, dtype=dt, stream=s)
        elif a.op == "mass":
            h.apply_mass(x, y, stream=s)
        elif a.op == "fmg":
            h.solve(x, y, precond=fe.FE_PC_FMG, max_it=a.cycles, stream=s)
        else:
            h.vcycle(x, y, dtype=dt, stream=s)
        e1.record(s)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    print(f"{a.op} P{a.degree} N={a.N} {a.dtype}: n={n} cells={h.n_cells()} ms/launch={np.mean(ms):.4f} "
          f"(min {np.min(ms):.4f})")
    h.close()


if __name__ == "__main__":
    main()
