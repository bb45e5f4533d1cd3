"""Single hot-path workloads for kernel profiling (ncu) and quick timing.

Each case assembles one 2D problem (`inputs.helmholtz_2d`), runs the call
once untimed (first-use costs), then `--reps` times inside an NVTX range
named "profiled", so a profiler can restrict itself to those launches:

    python -m paper_2209_14740_gb300.profile_cases matvec --g 511 --s 6 --r 3
    ncu --clock-control none --nvtx --nvtx-include "profiled/" --metrics gpu__time_duration.sum ...
        python -m paper_2209_14740_gb300.profile_cases solve --mode mixed

Cases: matvec (the SG operator), precond (the mean-value preconditioner),
solve (one preconditioned GMRES solve), cgs2 (the two CGS2 passes of Arnoldi
step --step of the flexible complex64 cycles, on a zeroed workspace).  Prints one JSON line with the
CUDA-event time per repetition (meaningless under a profiler).
"""
from __future__ import annotations

import argparse
import contextlib
import json

from . import binding as B
from . import inputs


@contextlib.contextmanager
def _nvtx(torch, name):
    try:
        torch.cuda.nvtx.range_push(name)
        pushed = True
    except Exception:   # profiling ranges are optional
        pushed = False
    try:
        yield
    finally:
        if pushed:
            torch.cuda.nvtx.range_pop()


def main(argv=None):
    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["matvec", "precond", "solve", "cgs2"])
    ap.add_argument("--dim", type=int, default=2, choices=[1, 2], help="1: the 1D workload with --g unknowns")
    ap.add_argument("--g", type=int, default=127)
    ap.add_argument("--s", type=int, default=3)
    ap.add_argument("--r", type=int, default=3)
    ap.add_argument("--kbar", type=float, default=30.0)
    ap.add_argument("--sigma", type=float, default=0.15)
    ap.add_argument("--prec", choices=["fp32", "fp64", "tf32", "fp16"], default="fp32",
                    help="matvec/precond precision (tf32 / fp16: the TF32 or binary16 fast-diagonalisation "
                         "preconditioner, 2D only)")
    ap.add_argument("--mode", choices=["mixed", "fp64", "fp32"], default="mixed", help="solve precision")
    ap.add_argument("--restart", type=int, default=50)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--inner-tol", type=float, default=0.0, help="mixed solve: inner reduction per refinement")
    ap.add_argument("--step", type=int, default=10, help="cgs2: Arnoldi step j of the timed passes")
    ap.add_argument("--tile-n", type=int, default=-1,
                    help="transform tile width to set (64, 128, 256; 0: built-in rule); default: as tuned")
    a = ap.parse_args(argv)

    B.load()
    dev = torch.device("cuda", 0)
    if a.dim == 1:
        op = B.SG(inputs.helmholtz_1d_c1(n_unknowns=a.g, r=a.r))
    else:
        op = B.SG(inputs.helmholtz_2d(a.g, a.s, a.r, a.kbar, a.sigma))
    if a.tile_n >= 0:
        t = op.tune_get()
        t["tc_tile_n"] = a.tile_n
        op.tune_set(t)
    prec = {"fp32": B.FP32, "fp64": B.FP64, "tf32": B.TF32, "fp16": B.FP16}[a.prec]
    cdt = torch.complex128 if prec == B.FP64 else torch.complex64
    gen = torch.Generator(device=dev).manual_seed(0)
    if a.case == "solve":
        b = torch.empty(op.N, dtype=torch.complex128, device=dev)
        op.rhs(b, B.FP64)
        x = torch.zeros_like(b)
        mode = {"mixed": B.MIXED, "fp64": B.FP64, "fp32": B.FP32}[a.mode]
        if mode == B.FP32:
            b = b.to(torch.complex64)
            x = torch.zeros_like(b)

        def call():
            return op.gmres(b, x, restart=a.restart, tol=1e-8 if mode != B.FP32 else 1e-5, prec=B.PREC_MEAN,
                            mode=mode, inner_tol=a.inner_tol)
    elif a.case == "cgs2":
        op.cgs2_pass(a.step, 0, restart=max(a.restart, a.step + 1))

        def call():
            op.cgs2_pass(a.step, 1)
            op.cgs2_pass(a.step, 2)
    else:
        X = torch.randn(op.N, dtype=cdt, device=dev, generator=gen)
        Y = torch.empty_like(X)
        if a.case == "matvec":
            def call():
                op.matvec(X, Y, B.FP32 if prec in (B.TF32, B.FP16) else prec)
        else:
            def call():
                op.precond(X, Y, B.PREC_MEAN, prec)
    out = call()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    with _nvtx(torch, "profiled"):
        e0.record(stream)
        for _ in range(a.reps):
            out = call()
        e1.record(stream)
        torch.cuda.synchronize()
    line = {"case": a.case, "g": a.g, "s": a.s, "r": a.r, "P": op.P, "N": op.N, "reps": a.reps,
            "ms_per_rep": e0.elapsed_time(e1) / max(a.reps, 1)}
    if isinstance(out, dict):
        line.update(iters=out["iters"], outer=out["outer"], relres=out["relres"])
    print(json.dumps(line))
    op.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
