#!/usr/bin/env python
"""Benchmark of the SG Helmholtz GMRES hot path on GB300.

Headline (`value`): SG-GMRES solves per second to relative residual 1e-8
(||b - A x|| / ||b|| computed in FP64) on the largest single-GPU workload:
511 x 511 nodes (h = 1/510), absorbing boundary,
k = 60 (1 + 0.1 sum_{l<=6} l^-1 cos(l pi x) cos(l pi y) xi_l), Legendre chaos
of total degree 3 in 6 variables (P = 84), Gaussian source at the centre:
21,934,164 complex unknowns.  The timed step is one full solve of the
mixed-precision path (complex64 GMRES(30) cycles inside FP64 iterative
refinement, mean-value preconditioner, zero initial guess) with b resident
in HBM.  The preconditioner set-up (once per system, in sg_assemble) is
reported separately as setup_ms.

Beside it the line reports: the plain FP64 GPU GMRES(30) on the same system
(`fp64`, with the FP64 kernels against the measured FP64 FMA rate), the error
of every mixed result against an FP64 GPU solve to 1e-12 (`error`), the
end-to-end number through the C ABI with host buffers (`e2e`), the roofline
of the dominant kernel (`roofline`: the tensor-core transform) and of CGS2
pass 2 (`roofline_cgs2`, HBM), the SG matvec bandwidth (`matvec`), the
127 x 127 workload (`cfg2_127`), the 1D workload, the batched and learned
warm-start legs, clocks sampled during the timed region, and the CPU oracle
(`cpu_baseline`) on a bounded sample.

--impl reference times the CPU oracle (oracle/, plain FP64 NumPy/SciPy) on
the same metric: each step a bounded sample (Arnoldi steps of its GMRES(30)
on the 127 x 127 member of the workload family), extrapolated as stated in
the line.

Multi-GPU: the solves are independent (replicas only): each rank solves its
own copy, value = total solves / max rank time, scaling "weak".
"""
from __future__ import annotations

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

METRIC = ("SG-GMRES solves/s to rel.res 1e-8 (mixed precision: complex64 GMRES(30) in FP64 refinement, "
          "mean-value preconditioner)")
UNIT = "solves/s"
WORKLOAD = {"workload": "helmholtz_2d_511x511_s6_deg3", "nodes": "511x511", "h": "1/510", "s": 6, "degree": 3,
            "P": 84, "unknowns": 21934164, "kbar": 60.0, "sigma": 0.1, "restart": 30, "tol": 1e-8,
            "preconditioner": "mean-value I(x)S(xi_bar)", "source": "gaussian w=0.02 at (0.5,0.5)"}
MATVEC_WORKLOAD = "helmholtz_2d_511x511_s6_deg3 (P=84, 21,934,164 unknowns)"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the
# generated complex64 operator kernel at 511 x 511, P = 84, from an earlier ncu
# capture (the matvec summary under profiles/), not measured live by this
# script.  Reported only while the generator still emits this kernel source and
# tile (SHA-256 below): a changed kernel reports null.
MATVEC_TRAFFIC = {"sha256": "0e5a4679d2e0f084f9f73ce6af95304f6010fe7044be5c825df92d9d73acfd2d",
                  "bytes": 183150592 + 123807488}
# DRAM bytes of one launch of the binary16 transform (transform 2 of an apply
# at 511 x 511, P = 84) from the ncu captures summarised under profiles/: the
# persistent k_tc_cgemm_ps<128, true> ("ps") and the paired 256-column
# k_tc_hgemm_w ("wide"); each reported while its kernel source (the section
# of k_tc_gemm.cu between the markers, SHA-256 below) is unchanged.
TRANSFORM_TRAFFIC = {
    "ps": {"begin": "template <int BN>\nstruct CfgP", "end": "// ------------------------------------------------------------------ paired 256-column",
           "sha256": "17314e41f33bc6264a05f8d99e050307a6d6ddc102cc9323a472040d7ea71198", "bytes": 92218112 + 47893248},
    "wide": {"begin": "// ------------------------------------------------------------------ paired 256-column",
             "end": "// Check of the bounded wait",
             "sha256": "1c3a2958e35b2ae42c1747348c4c3e41e19dee986912c16e3e35e11f04f0d9ed", "bytes": 92444160 + 47176192},
}
# Arnoldi step of the CGS2 passes timed for their roofline (the step of the
# traffic capture below; the 511^2 solve's 41 steps have mean index 6.4)
CGS2_STEP = 10
# DRAM bytes of one launch of CGS2 pass 2 on the binary16 basis (k_hb_second,
# step 10) at 255^2, P = 84 (np_255 binary16 pairs per basis slot), from the
# ncu capture summarised under profiles/, scaled to the slot size np (every
# term of the pass's traffic is a multiple of the unknowns); reported while
# the pass's source (the section of solver.cu between the markers, SHA-256
# below) is unchanged.
CGS2_TRAFFIC = {"begin": "// Pass 2 on the binary16 basis", "end": "// r = b - Ax (or r = b when Ax",
                "sha256": "c603c346f722fbd04065f579f7bc9ad3039d8afb2e4c6289954f33d98c9790a7",
                "bytes": 285044736 + 17458688, "np": 84 * 255 * 256}
# Dense TF32 / BF16 tensor throughput, nominal (2D preconditioner transforms run on
# TF32 tensor cores; their peak is the measured BF16 peak times this ratio).
TF32_PER_BF16 = 1.1 / 2.25
# The oracle's sample: the 127 x 127 member of the workload family (same s,
# degree, kbar, sigma; N = 1,354,836), Arnoldi steps of its GMRES(30).
ORACLE_SAMPLE_G = 127
ORACLE_SAMPLE_STEPS = 10
# Arnoldi steps of the plain FP64 GPU GMRES(30) on the 511 x 511 system
# (measured on GB300, the `fp64.iterations` of the bench line: used by the
# reference arm, which runs without a GPU)
FP64_STEPS_511 = 33


def nvtx(torch, name):
    """Push an NVTX range (ncu --nvtx-include selects launches by it)."""
    try:
        torch.cuda.nvtx.range_push(name)
        return True
    except Exception:
        return False


def nvtx_pop(torch, pushed):
    if pushed:
        torch.cuda.nvtx.range_pop()


def matvec_traffic():
    import hashlib

    from paper_2209_14740_gb300 import codegen_matvec
    src = codegen_matvec.gen_kernel_tkp(6, 3)[2] + repr(codegen_matvec.PTILE_2D)
    digest = hashlib.sha256(src.encode()).hexdigest()
    return MATVEC_TRAFFIC["bytes"] if digest == MATVEC_TRAFFIC["sha256"] else None


def transform_section_sha(kind):
    import hashlib
    t = TRANSFORM_TRAFFIC[kind]
    src = open(os.path.join(ROOT, "paper_2209_14740_gb300", "csrc", "k_tc_gemm.cu")).read()
    i = src.find(t["begin"])
    j = src.find(t["end"], i + 1)
    if i < 0 or j < 0:
        return None
    return hashlib.sha256(src[i:j].encode()).hexdigest()


def transform_traffic(kind):
    t = TRANSFORM_TRAFFIC[kind]
    return t["bytes"] if t["sha256"] and transform_section_sha(kind) == t["sha256"] else None


def cgs2_section_sha():
    import hashlib
    src = open(os.path.join(ROOT, "paper_2209_14740_gb300", "csrc", "solver.cu")).read()
    i = src.find(CGS2_TRAFFIC["begin"])
    j = src.find(CGS2_TRAFFIC["end"], i + 1)
    if i < 0 or j < 0:
        return None
    return hashlib.sha256(src[i:j].encode()).hexdigest()


def cgs2_traffic(np_):
    t = CGS2_TRAFFIC
    if not t["sha256"] or not t["bytes"] or cgs2_section_sha() != t["sha256"]:
        return None
    return t["bytes"] * np_ / t["np"]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def load_tensor_peak(fp16=False):
    """Dense tensor TFLOP/s for TF32 (measured BF16 burst peak x nominal
    TF32/BF16 ratio) or binary16 (the BF16 peak itself: the same nominal rate)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    ratio = 1.0 if fp16 else TF32_PER_BF16
    how = "measured bf16 (binary16 runs at the bf16 rate)" if fp16 else "measured bf16 x nominal tf32/bf16"
    if os.path.exists(p):
        return float(json.load(open(p))["bf16_tflops"]) * ratio, how
    return 1900.0 * ratio, how.replace("measured", "fallback")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(gpus: int):
    from paper_2209_14740_gb300 import replicas
    return replicas.init()


def barrier(world):
    from paper_2209_14740_gb300 import replicas
    replicas.barrier(world)


def max_over_ranks(v: float, world: int) -> float:
    from paper_2209_14740_gb300 import replicas
    return replicas.max_over_ranks(v, world)


def oracle_sample_setup():
    """Assemble the oracle's explicit SG system of the sample (the 127 x 127
    member of the workload family) and factor its mean-value block once (as
    sg_assemble does on the GPU side)."""
    from oracle import krylov, sg
    from paper_2209_14740_gb300 import inputs
    pr = inputs.helmholtz_2d(ORACLE_SAMPLE_G, 6, 3, 60.0, 0.1)
    S = sg.assemble_problem(pr)
    return S, krylov.BlockPrecond(S.S0, S.P)


def oracle_sample_step_seconds(S, M, steps=ORACLE_SAMPLE_STEPS):
    """Mean seconds per Arnoldi step of the oracle's GMRES(30) (mean-value
    block preconditioner, CGS2, Givens) over the first `steps` steps of a
    cycle, plus its closing true-residual evaluation."""
    from oracle import krylov
    t0 = time.perf_counter()
    krylov.gmres(S.A, S.b, M, restart=30, tol=1e-300, maxit=steps)
    return (time.perf_counter() - t0) / steps


def oracle_extrapolate(step_s, n_sample, steps_511):
    """Oracle seconds per solve of the 511 x 511 system: step time x ratio of
    unknowns x Arnoldi steps of the solve.  The oracle's costs per step grow at
    least linearly in the unknowns (measured 63^2 -> 127^2 -> 255^2: 0.23,
    0.61, 2.69 s), and its CGS2 share grows with the step index, so this is an
    optimistic estimate of the oracle."""
    return step_s * (WORKLOAD["unknowns"] / n_sample) * steps_511


def oracle_sample_text(n_sample, steps_511, samples):
    return ("%d x %d Arnoldi steps of the oracle's GMRES(30) on the %dx%d member of the workload family "
            "(s=6, degree 3, kbar=60, sigma=0.1; N=%d), mean step time x %.2f (unknowns 511^2 / %d^2) x %d "
            "(Arnoldi steps of the FP64 solve of the 511^2 system); SuperLU single threaded, NumPy BLAS on all "
            "cores" % (samples, ORACLE_SAMPLE_STEPS, ORACLE_SAMPLE_G, ORACLE_SAMPLE_G, n_sample,
                       WORKLOAD["unknowns"] / n_sample, ORACLE_SAMPLE_G, steps_511))


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    S, M = oracle_sample_setup()
    n_sample = S.A.shape[0]
    for _ in range(args.warmup):
        oracle_sample_step_seconds(S, M)
    per_solve = [oracle_extrapolate(oracle_sample_step_seconds(S, M), n_sample, FP64_STEPS_511)
                 for _ in range(args.steps)]
    ms = 1000.0 * statistics.mean(per_solve)
    value = 1000.0 / ms
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": dict(WORKLOAD, oracle="NumPy/SciPy FP64 GMRES(30) + SuperLU block preconditioner",
                           world_size=world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": oracle_sample_text(n_sample, FP64_STEPS_511, args.steps)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line))
    return 0


def cfg1_leg(B, torch, dev):
    """1D workload (200 unknowns, Dirichlet / absorbing, k = 20 (1 + 0.1 xi),
    degree 5, P = 6, N = 1200), mean-value preconditioner, GMRES(100) to
    relres 1e-8 (latency bound: one solve is a few dozen tiny kernels).  Mixed
    precision (FP32 Arnoldi, FP64 refinement) and plain FP64; single solves
    replay CUDA graphs, the batch runs 256 copies concurrently (mixed)."""
    from paper_2209_14740_gb300 import inputs
    pr = inputs.helmholtz_1d_c1()
    op = B.SG(pr)
    b = torch.empty(op.N, dtype=torch.complex128, device=dev)
    op.rhs(b, B.FP64)
    x = torch.zeros_like(b)
    out = {"workload": "1D: 200 unknowns, k = 20(1 + 0.1 xi), degree 5 (P = 6, N = 1200), mean-value, "
                       "GMRES(100), tol 1e-8"}
    for name, mode in (("mixed", B.MIXED), ("fp64", B.FP64)):
        kw = dict(restart=100, tol=1e-8, prec=B.PREC_MEAN, mode=mode)
        for _ in range(3):
            info = op.gmres(b, x, **kw)
        torch.cuda.synchronize()
        reps = 50
        t1 = time.perf_counter()
        for _ in range(reps):
            info = op.gmres(b, x, **kw)
        torch.cuda.synchronize()
        out[name] = {"solves_per_s": reps / (time.perf_counter() - t1), "iterations": info["iters"],
                     "relres": info["relres"], "converged": bool(info["status"] == B.SG_OK)}
    kw = dict(restart=100, tol=1e-8, prec=B.PREC_MEAN, mode=B.MIXED)
    ops = [B.SG(pr) for _ in range(256)]
    bs = [b.clone() for _ in ops]
    xs = [torch.zeros_like(b) for _ in ops]
    B.gmres_batched(ops, bs, xs, **kw)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    st, inf = B.gmres_batched(ops, bs, xs, **kw)
    torch.cuda.synchronize()
    out["mixed_batched_256_solves_per_s"] = len(ops) / (time.perf_counter() - t1)
    out["batched_all_converged"] = bool(st == B.SG_OK)
    for o in ops:
        o.close()
    op.close()
    return out


def learned_leg(args, B, torch, dev):
    """Warm-start workload: (kbar, sigma, lc, x_s, y_s) uniform in [10,40] x
    [0.05,0.2] x [0.1,0.5] x [0.2,0.8]^2 on 127x127, s=3, degree 3 (N=322,580).
    Trains on `--learned-train` solved problems, then solves `--learned-test`
    held-out problems: mixed + learned guess + batched against plain FP64 one
    at a time."""
    import numpy as np

    from paper_2209_14740_gb300 import inputs, warmstart

    ptrain = inputs.warmstart_params(1, args.learned_train)
    ptest = inputs.warmstart_params(2, args.learned_test)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S, its_train = warmstart.solve_batch(ptrain, torch, dev, tol=1e-10)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    ws = warmstart.build(ptrain, S, torch, dev, rank=64, n_snapshots=min(1024, len(ptrain)), epochs=300, batch=64)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    # POD ceiling: the best any rank-R decoder can do on the held-out set
    U256, lam = warmstart.pod_basis(S, 256, min(1024, len(ptrain)), torch, dev)
    del S
    ops = [B.SG(inputs.warmstart_problem(p)) for p in ptest]
    bs = []
    for op in ops:
        bb = torch.empty(op.N, dtype=torch.complex128, device=dev)
        op.rhs(bb, B.FP64)
        bs.append(bb)
    xs = [torch.zeros_like(bb) for bb in bs]
    kw = dict(restart=50, tol=1e-8, prec=B.PREC_MEAN, maxit=20000)

    def zero_batched():
        return B.gmres_batched(ops, bs, xs, mode=B.MIXED, **kw)

    # the guesses go to one buffer that every call reuses: the batched solve's
    # graph is keyed by its vectors, so it is built once
    x0buf = torch.empty((len(ops), ops[0].N), dtype=torch.complex128, device=dev)
    x0list = [x0buf[k] for k in range(len(ops))]

    def learned_batched():
        ws.model.predict(ptest, x0buf)
        return B.gmres_batched(ops, bs, xs, x0s=x0list, x0_policy=B.X0_SCALED, mode=B.MIXED, **kw), x0buf

    zero_batched()                                                 # workspaces
    learned_batched()                                              # first use of the inference kernels
    timings = {}
    for name, fn in (("zero", zero_batched), ("learned", learned_batched)):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        timings[name] = (time.perf_counter() - t1, out)
    (st_z, inf_z) = timings["zero"][1]
    (st_l, inf_l), x0 = timings["learned"][1]
    ws.model.predict(ptest, x0buf)                                 # the unscaled guesses again
    rel = [float(torch.linalg.norm(x0buf[k] - xs[k]) / torch.linalg.norm(xs[k])) for k in range(len(ops))]
    graph_steps = sum(i["graph_outer"] for i in inf_l)
    del x0, x0buf, x0list
    Xt = torch.stack([v.to(torch.complex64) for v in xs]).contiguous()
    ceil = warmstart.pod_errors(U256, Xt, (64, 128, 256), torch, dev)
    lam_pos = np.clip(lam, 0.0, None)
    pod_ceiling = {str(R): {"relerr_median": float(np.median(e)), "relerr_max": float(np.max(e)),
                            "train_energy": float(lam_pos[:R].sum() / lam_pos.sum())} for R, e in ceil.items()}
    del Xt, U256
    for op, bb in zip(ops, bs):                                    # FP64 workspaces (one iteration each)
        op.gmres(bb, torch.zeros_like(bb), mode=B.FP64, restart=50, tol=1e-8, prec=B.PREC_MEAN, maxit=1)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    inf_s = [op.gmres(bb, torch.zeros_like(bb), mode=B.FP64, **kw) for op, bb in zip(ops, bs)]
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t1
    for op in ops:
        op.close()
    n = len(ops)
    return {"workload": "warm-start family: kbar~U[10,40], sigma~U[0.05,0.2], lc~U[0.1,0.5], source~U[0.2,0.8]^2; "
                        "127x127, s=3, degree 3 (N=322,580); GMRES(50), mean-value, tol 1e-8",
            "train_problems": len(ptrain), "test_problems": n,
            "train_data_s": t_data, "train_iterations_mean": float(np.mean(its_train)),
            "fit_s": t_train, "fit_breakdown_s": ws.timings, "pod_rank": ws.rank, "pod_energy": ws.energy_captured,
            "loss_first_last": [ws.loss_history[0], ws.loss_history[-1]],
            "guess_relerr_median": float(np.median(rel)),
            "pod_ceiling_heldout": pod_ceiling,
            "iterations_mean_zero": float(np.mean([i["iters"] for i in inf_z])),
            "iterations_mean_learned": float(np.mean([i["iters"] for i in inf_l])),
            "mixed_batched_zero_solves_per_s": n / timings["zero"][0],
            "mixed_batched_learned_solves_per_s": n / timings["learned"][0],
            "learned_batched_route": "one graph launch with the guesses, %d of %d refinement steps inside it" % (
                graph_steps, sum(i["outer"] for i in inf_l)),
            "fp64_sequential_solves_per_s": n / t_seq,
            "speedup_vs_fp64_sequential": t_seq / timings["learned"][0],
            "all_converged": bool(st_z == B.SG_OK and st_l == B.SG_OK and all(i["status"] == B.SG_OK for i in inf_s)
                                  and all(i["relres"] <= 1e-8 for i in inf_l))}


def timed_solves(op, b, x, steps, flush, stream, torch, **kw):
    """`steps` solves, each timed with CUDA events on `stream`, L2 flushed
    before each."""
    times, infos = [], []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = op.gmres(b, x, **kw)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        infos.append(info)
    return times, infos


def event_ms(torch, stream, fn, reps):
    """Mean milliseconds of fn() over reps calls, CUDA events on `stream`."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def rel_err(torch, a, ref):
    return float(torch.linalg.vector_norm(a - ref) / torch.linalg.vector_norm(ref))


def cfg2_leg(B, torch, dev, flush, stream):
    """127 x 127, s = 3, degree 3 (P = 20, N = 322,580): mixed GMRES(50) and
    plain FP64 GMRES(50), mean-value preconditioner, tol 1e-8."""
    from paper_2209_14740_gb300 import inputs
    op = B.SG(inputs.config_2d_127())
    b = torch.empty(op.N, dtype=torch.complex128, device=dev)
    op.rhs(b, B.FP64)
    x = torch.zeros_like(b)
    out = {"workload": "helmholtz_2d_127x127_s3_deg3 (P=20, N=322,580), GMRES(50), mean-value, tol 1e-8"}
    for name, mode, reps in (("mixed", B.MIXED, 10), ("fp64", B.FP64, 3)):
        kw = dict(restart=50, tol=1e-8, prec=B.PREC_MEAN, mode=mode)
        for _ in range(3):
            op.gmres(b, x, **kw)
        t, inf = timed_solves(op, b, x, reps, flush, stream, torch, **kw)
        ms = statistics.mean(t)
        out[name] = {"ms": ms, "solves_per_s": 1000.0 / ms, "iterations": inf[-1]["iters"],
                     "outer": inf[-1]["outer"], "relres": inf[-1]["relres"],
                     "converged": all(i["status"] == B.SG_OK for i in inf)}
    out["mixed_speedup_vs_fp64"] = out["fp64"]["ms"] / out["mixed"]["ms"]
    op.close()
    return out


def batched_leg(B, torch, dev):
    """64 heterogeneous systems (g ~ U{63..255}, kbar ~ U[10,40], sigma ~
    U[0.05,0.2], s ~ U{2,3,4}, degree ~ U{2,3}): mixed batched solve against
    plain FP64 one at a time."""
    from paper_2209_14740_gb300 import inputs
    probs = inputs.batch_64()
    ops = [B.SG(p) for p in probs]
    bs = []
    for op in ops:
        bb = torch.empty(op.N, dtype=torch.complex128, device=dev)
        op.rhs(bb, B.FP64)
        bs.append(bb)
    xs = [torch.zeros_like(bb) for bb in bs]
    kw = dict(restart=30, tol=1e-8, prec=B.PREC_MEAN, maxit=20000)
    B.gmres_batched(ops, bs, xs, mode=B.MIXED, **kw)          # warm-up (workspaces, graph instantiation)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    st_b, inf_b = B.gmres_batched(ops, bs, xs, mode=B.MIXED, **kw)
    torch.cuda.synchronize()
    t_batched = time.perf_counter() - t1
    ok_b = st_b == B.SG_OK and all(i["relres"] <= 1e-8 for i in inf_b)
    # the per-system route (host thread pool, one stream per system)
    B.gmres_batched(ops, bs, xs, mode=B.MIXED, concurrency=-1, **kw)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    st_p, inf_p = B.gmres_batched(ops, bs, xs, mode=B.MIXED, concurrency=-1, **kw)
    torch.cuda.synchronize()
    t_pool = time.perf_counter() - t1
    ok_b = ok_b and st_p == B.SG_OK and [i["iters"] for i in inf_p] == [i["iters"] for i in inf_b]
    for op, bb, xx in zip(ops, bs, xs):                        # warm-up of the FP64 workspaces
        op.gmres(bb, xx, mode=B.FP64, **kw)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    inf_s = [op.gmres(bb, xx, mode=B.FP64, **kw) for op, bb, xx in zip(ops, bs, xs)]
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t1
    ok_s = all(i["status"] == B.SG_OK for i in inf_s)
    from paper_2209_14740_gb300 import tune_table
    n_tuned = sum(1 for op in ops if tune_table.lookup(op.info["dim"], op.info["mx"], op.info["my"], op.info["s"],
                                                       op.info["r"]) is not None)
    out = {"systems": len(ops), "systems_with_tuned_shapes": n_tuned,
           "workload": "64 systems: g ~ U{63..255}, kbar ~ U[10,40], "
           "sigma ~ U[0.05,0.2], s ~ U{2,3,4}, degree ~ U{2,3} (P 6-35), GMRES(30), mean-value",
           "unknowns_total": int(sum(op.N for op in ops)),
           "mixed_batched_solves_per_s": len(ops) / t_batched,
           "mixed_batched_route": "one graph launch, %d of %d refinement steps inside it" % (
               sum(i["graph_outer"] for i in inf_b), sum(i["outer"] for i in inf_b)),
           "mixed_per_system_route_solves_per_s": len(ops) / t_pool,
           "fp64_sequential_solves_per_s": len(ops) / t_seq,
           "speedup_vs_fp64_sequential": t_seq / t_batched,
           "all_converged": bool(ok_b and ok_s),
           "iterations_mixed_total": int(sum(i["iters"] for i in inf_b)),
           "iterations_fp64_total": int(sum(i["iters"] for i in inf_s))}
    for op in ops:
        op.close()
    return out


def run_ours(args):
    import torch

    from paper_2209_14740_gb300 import binding, inputs, replicas

    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    B = binding
    B.load()

    # ---------------------------------------------------------------- set-up
    pr = inputs.config_2d_511()
    t0 = time.perf_counter()
    op = B.SG(pr)
    torch.cuda.synchronize()
    setup_ms = 1000 * (time.perf_counter() - t0)
    # launch shapes in effect: the committed sg_autotune table's entry for
    # this size (applied by SG), else the built-in rules
    from paper_2209_14740_gb300 import tune_table
    tuning = {"source": "tune_table.json (sg_autotune on GB300)" if tune_table.lookup(
        op.info["dim"], op.info["mx"], op.info["my"], op.info["s"], op.info["r"]) else "built-in rules"}
    tuning.update({k: v for k, v in op.tune_get().items() if k in B.TUNE_KEYS})
    N, n, P = op.N, op.n, op.P
    info_h = op.info
    b = torch.empty(N, dtype=torch.complex128, device=dev)
    op.rhs(b, B.FP64)
    x = torch.zeros_like(b)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2 (129 MB)
    solve = dict(restart=30, tol=1e-8, prec=B.PREC_MEAN, mode=B.MIXED, maxit=3000)

    for _ in range(args.warmup):
        op.gmres(b, x, **solve)
    torch.cuda.synchronize()

    # ---------------------------------------------------------------- timed region
    barrier(world)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    if rank == 0:
        clk.start()
    l0 = B.kernel_launches()
    pushed = nvtx(torch, "timed")
    times, infos = timed_solves(op, b, x, args.steps, flush, stream, torch, **solve)
    launches = B.kernel_launches() - l0
    nvtx_pop(torch, pushed)
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop() if rank == 0 else None
    ms = max_over_ranks(statistics.mean(times), world)
    value = replicas.whole_job_rate(1.0, ms / 1000.0, world)   # one solve per step per rank
    ok = all(i["status"] == B.SG_OK and i["relres"] <= 1e-8 for i in infos)
    x_mixed = x.clone()

    # ---------------------------------------------------------------- dominant kernel of the step
    # The preconditioner apply of the solve's complex64 cycles is four
    # launches of the tensor-core transform kernel, complex GEMMs of (P my) x
    # mx by mx x mx (x direction) and (P mx) x my by my x my (y direction).
    # On the binary16 route every Arnoldi step after the first of a cycle
    # runs all four as binary16 GEMMs by tensor copies (transform 1 from the
    # binary16 copy of the basis vector that the second CGS2 pass writes):
    # the paired 256-column kernel k_tc_hgemm_w where the tuning selects it,
    # else the persistent k_tc_cgemm_ps; the first step of a cycle (and
    # sg_precond) runs transform 1 in TF32 from the complex64 vector.  The
    # dominant kernel is timed alone through sg_fd_transform (transform 2,
    # the same launch as inside the apply), 20 launches with CUDA events on
    # the solve's stream; transforms 3 and 4, the whole apply and the TF32
    # transform 1 beside it.
    top = None
    cgs = None
    if info_h.get("tf32_route"):
        mx, my = info_h["mx"], info_h["my"]
        f16 = bool(info_h.get("fp16_route")) and not op.tune_get().get("tf32_transforms")
        if f16:
            mxp, myp = (mx + 3) // 4 * 4, (my + 3) // 4 * 4
        else:
            mxp, myp = mx + (mx & 1), my + (my & 1)
        form = B.FP16 if f16 else B.TF32
        reps = 20
        Xp = torch.randn(N, dtype=torch.complex64, device=dev)
        Zp = torch.empty_like(Xp)
        for _ in range(3):
            op.precond(Xp, Zp, B.PREC_MEAN, form)
        pushed = nvtx(torch, "precond")
        t_apply = event_ms(torch, stream, lambda: op.precond(Xp, Zp, B.PREC_MEAN, form), reps)
        nvtx_pop(torch, pushed)
        del Xp, Zp
        size = P * max(mx, my) * max(mxp, myp)
        T1 = torch.randn(size, dtype=torch.complex64, device=dev)
        if f16:
            T1.zero_()
        T2 = torch.empty_like(T1)
        for _ in range(3):
            op.fd_transform(1, T1, T2, B.PREC_MEAN, form)
            op.fd_transform(0, T1, T2, B.PREC_MEAN, form)
        t_ps = event_ms(torch, stream, lambda: op.fd_transform(1, T1, T2, B.PREC_MEAN, form), reps)
        t_t3 = event_ms(torch, stream, lambda: op.fd_transform(2, T2, T1, B.PREC_MEAN, form), reps)
        Yp = torch.empty(N, dtype=torch.complex64, device=dev)
        t_t4 = event_ms(torch, stream, lambda: op.fd_transform(3, T1, Yp, B.PREC_MEAN, form), reps)
        del Yp
        t_t1 = event_ms(torch, stream, lambda: op.fd_transform(0, T1, T2, B.PREC_MEAN, form), reps)
        del T1, T2
        flops = 8.0 * P * mx * my * my           # transform 2: (P mx) x my by my x my, complex
        peak_t, peak_kind_t = load_tensor_peak(fp16=f16)
        peak_tf32, _ = load_tensor_peak(fp16=False)
        ach = flops / (t_ps * 1e-3) / 1e12
        wide = f16 and op.tune_get().get("tc_tile_n") == 256
        tr = transform_traffic("wide" if wide else "ps") if f16 else None
        if wide:
            kname = ("k_tc_hgemm_w (paired 256-column binary16 transform, kind::f16, clusters of two CTAs "
                     "sharing B stages by multicast copies; all 4 launches of the apply in the cycles' steps "
                     "after the first, 3 of 4 in the first)")
            tsrc = "ncu capture of this kernel source at 511x511, P = 84 (its summary under profiles/)"
        elif f16:
            kname = ("k_tc_cgemm_ps<%d, true> (persistent binary16 transform, kind::f16; all 4 launches of the "
                     "apply in the cycles' steps after the first, 3 of 4 in the first)" % op.tune_get().get("tc_tile_n"))
            tsrc = "ncu capture of this kernel source at 511x511, P = 84 (its summary under profiles/)"
        else:
            kname = "k_tc_cgemm_ps (persistent plain-TF32 transform, 3 of the 4 launches per apply)"
            tsrc = None
        top = {"kernel": kname, "bound": "tensor",
               "achieved": ach, "peak": peak_t, "unit": "TFLOP/s", "frac": ach / peak_t, "traffic": tr,
               "traffic_source": tsrc if tr else None,
               "peak_kind": peak_kind_t, "us_per_launch": 1000.0 * t_ps, "flops_per_launch": flops,
               "units": "8 P m^3 real flop per launch (complex GEMM of (P m) x m by m x m; m = 511, P = 84)",
               "transform3_us": 1000.0 * t_t3, "transform4_us": 1000.0 * t_t4,
               "frac_mean_of_transforms_2_to_4": flops / (statistics.mean([t_ps, t_t3, t_t4]) * 1e-3) / 1e12 / peak_t,
               "transform1_complex64_input_us": 1000.0 * t_t1,
               "transform1_complex64_input_frac_tf32": flops / (t_t1 * 1e-3) / 1e12 / peak_tf32,
               "apply_ms": t_apply}
        # The CGS2 passes of one Arnoldi step of the flexible cycles, the
        # step's largest kernels (pass 2 the largest share of the solve):
        # step j = CGS2_STEP on a zeroed workspace through sg_cgs2_pass (the
        # form the mixed solver runs: on the binary16 route the binary16
        # basis), 20 launches each with CUDA events on the solve's stream
        # (each preceded by the pass's 64-byte clear of the done flag).
        # Algorithmic bytes with the binary16 basis (np pairs per slot, the
        # padded rows): pass 1 reads slots 0..j and w (complex64); pass 2
        # reads the same and writes slot j+1.  With the complex64 basis: pass
        # 1 reads V_0..V_j and w, pass 2 reads V_0..V_j and w and writes w.
        jc = CGS2_STEP
        op.cgs2_pass(jc, 0, restart=solve["restart"])
        for _ in range(3):
            op.cgs2_pass(jc, 1)
            op.cgs2_pass(jc, 2)
        t_p1 = event_ms(torch, stream, lambda: op.cgs2_pass(jc, 1), reps)
        t_p2 = event_ms(torch, stream, lambda: op.cgs2_pass(jc, 2), reps)
        np_ = P * my * ((mx + 3) // 4 * 4)
        if f16:
            b_p1 = (jc + 1) * np_ * 4 + N * 8
            b_p2 = (jc + 1) * np_ * 4 + N * 8 + np_ * 4
            b_model = 2 * (jc + 1) * np_ * 4
            kname = ("k_hb_second (CGS2 pass 2 of a flexible Arnoldi step on the binary16 basis, j = %d: "
                     "projection update, the new slot in binary16 and its norm, Givens column)" % jc)
            units = "(j + 2) np 4 B + N 8 B per launch (binary16 slots of np pairs), j = %d, np = %d, N = %d" % (
                jc, np_, N)
        else:
            b_p1 = (jc + 2) * N * 8
            b_p2 = (jc + 2) * N * 8 + N * 8
            b_model = 2 * (jc + 1) * N * 8
            kname = "k_cgs2_second<float> (CGS2 pass 2 of a flexible complex64 Arnoldi step, j = %d)" % jc
            units = "(j + 3) N 8 B per launch, j = %d, N = %d" % (jc, N)
        hbm_peak, hbm_kind = load_peaks()
        tr2 = cgs2_traffic(np_) if f16 else None
        cgs = {"kernel": kname, "bound": "hbm", "achieved": b_p2 / (t_p2 * 1e-3) / 1e9, "peak": hbm_peak,
               "unit": "GB/s", "frac": b_p2 / (t_p2 * 1e-3) / 1e9 / hbm_peak, "traffic": tr2,
               "traffic_source": ("ncu capture of this kernel source at 255^2 (P = 84), step %d, scaled by "
                                  "the slot size (its summary under profiles/)" % jc) if tr2 else None,
               "peak_kind": hbm_kind, "us_per_launch": 1000.0 * t_p2, "bytes_per_launch": b_p2, "units": units,
               "pass1": {"kernel": "k_hb_dots" if f16 else "k_cgs_dots<float>", "us_per_launch": 1000.0 * t_p1,
                         "bytes_per_launch": b_p1, "gbs": b_p1 / (t_p1 * 1e-3) / 1e9,
                         "frac": b_p1 / (t_p1 * 1e-3) / 1e9 / hbm_peak},
               "both_passes_basis_model_frac": b_model / ((t_p1 + t_p2) * 1e-3) / 1e9 / hbm_peak}

    # ---------------------------------------------------------------- end to end with host buffers
    bh = torch.empty(N, dtype=torch.complex128, pin_memory=True)
    bh.copy_(b)
    xh = torch.empty(N, dtype=torch.complex128, pin_memory=True)
    for _ in range(max(1, min(args.warmup, 2))):
        op.gmres(bh.numpy(), xh.numpy(), host_io=True, **solve)
    torch.cuda.synchronize()
    te = []
    for _ in range(max(2, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ie = op.gmres(bh.numpy(), xh.numpy(), host_io=True, **solve)
        te.append(time.perf_counter() - t1)
        assert ie["status"] == B.SG_OK
    e2e_ms = 1000 * statistics.mean(te)
    x_e2e = torch.from_numpy(xh.numpy()).to(dev)
    del bh, xh

    # ---------------------------------------------------------------- plain FP64 GPU GMRES, same system
    fp64_kw = dict(solve, mode=B.FP64)
    op.gmres(b, torch.zeros_like(b), **dict(fp64_kw, maxit=1))       # FP64 workspace
    x64 = torch.zeros_like(b)
    t64, i64 = timed_solves(op, b, x64, 2 if not args.quick else 1, flush, stream, torch, **fp64_kw)
    fp64_ms = statistics.mean(t64)
    # reference solution for the error of every result: FP64 GPU GMRES(30) to 1e-12
    x_ref = torch.zeros_like(b)
    i_ref = op.gmres(b, x_ref, **dict(fp64_kw, tol=1e-12))
    error = {"reference": "FP64 GPU GMRES(30) to relres 1e-12 (relres %.2e, %d Arnoldi steps)"
                          % (i_ref["relres"], i_ref["iters"]),
             "mixed": rel_err(torch, x_mixed, x_ref), "mixed_e2e": rel_err(torch, x_e2e, x_ref),
             "fp64_tol_1e-8": rel_err(torch, x64, x_ref)}
    del x_e2e

    # FP64 kernels against the measured FP64 FMA rate of this GPU
    fp64_peak = B.alu_peak(True)
    fp32_peak = B.alu_peak(False)
    X64 = torch.randn(N, dtype=torch.complex128, device=dev)
    Z64 = torch.empty_like(X64)
    op.precond(X64, Z64, B.PREC_MEAN, B.FP64)
    t_ap64 = event_ms(torch, stream, lambda: op.precond(X64, Z64, B.PREC_MEAN, B.FP64), 3)
    mx, my = info_h["mx"], info_h["my"]
    fl_ap64 = 2 * 8.0 * P * my * mx * mx                     # the two x eigen-transforms (complex GEMMs)
    op.matvec(X64, Z64, B.FP64)
    t_mv64 = event_ms(torch, stream, lambda: op.matvec(X64, Z64, B.FP64), 3)
    fl_mv64 = 4.0 * (info_h["coupling_nnz"] + 5 * P) * n    # real x complex products of a row, interior nodes
    del X64, Z64
    fp64 = {"solves_per_s": 1000.0 / fp64_ms, "ms": fp64_ms, "iterations": i64[-1]["iters"],
            "relres": i64[-1]["relres"], "mixed_speedup": fp64_ms / ms * world,
            "fp64_fma_peak_tflops": fp64_peak, "fp32_fma_peak_tflops": fp32_peak,
            "precond_apply": {"ms": t_ap64, "flops": fl_ap64,
                              "tflops": fl_ap64 / (t_ap64 * 1e-3) / 1e12,
                              "frac_of_fp64_peak": fl_ap64 / (t_ap64 * 1e-3) / 1e12 / fp64_peak,
                              "note": "two complex FP64 eigen-transforms (k_cgemm<double>, 8 P m^3 flop each) plus "
                                      "the pivoted y sweeps, whose time is included (a lower bound on the GEMMs' rate)"},
            "operator": {"ms": t_mv64, "flops": fl_mv64, "tflops": fl_mv64 / (t_mv64 * 1e-3) / 1e12,
                         "frac_of_fp64_peak": fl_mv64 / (t_mv64 * 1e-3) / 1e12 / fp64_peak,
                         "gbs": (N * 16 * 2 + (pr.s + 1) * n * 8) / (t_mv64 * 1e-3) / 1e9,
                         "note": "4 (nnz of the P x P coupling + 5 P) flop per grid point"}}

    # ---------------------------------------------------------------- matvec bandwidth (dominant HBM kernel)
    mv = None
    if rank == 0 and not args.skip_matvec:
        g = torch.Generator(device=dev).manual_seed(0)
        X = torch.randn(N, dtype=torch.complex64, device=dev, generator=g)
        Y = torch.empty_like(X)
        for _ in range(3):
            op.matvec(X, Y, B.FP32)
        torch.cuda.synchronize()
        reps = 20
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
        for k in range(reps):
            flush.zero_()
            ev[2 * k].record(stream)
            op.matvec(X, Y, B.FP32)
            ev[2 * k + 1].record(stream)
        torch.cuda.synchronize()
        t_mv = statistics.mean(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(reps))
        bytes_mv = N * 8 * 2 + (pr.s + 1) * n * 4
        peak, peak_kind = load_peaks()
        mv = {"workload": MATVEC_WORKLOAD, "dtype": "c64", "ms": t_mv, "bytes": bytes_mv,
              "gbs": bytes_mv / (t_mv * 1e-3) / 1e9, "peak_gbs": peak, "peak_kind": peak_kind}
        tr = matvec_traffic()
        mv["roofline"] = {"kernel": "k_mvkp_s6r3<32, 4> (SG operator, complex64, 511x511 P=84)", "bound": "hbm",
                          "achieved": mv["gbs"], "peak": peak, "unit": "GB/s", "frac": mv["gbs"] / peak,
                          "traffic": tr, "traffic_source": "earlier ncu capture of this kernel source" if tr else None,
                          "peak_kind": peak_kind}
        del X, Y
    op.close()
    del b, x, x64, x_ref, x_mixed
    torch.cuda.empty_cache()

    # ---------------------------------------------------------------- the other workloads
    cfg2 = batched = cfg1 = learned = None
    if rank == 0 and not args.skip_configs:
        cfg2 = cfg2_leg(B, torch, dev, flush, stream)
        cfg1 = cfg1_leg(B, torch, dev)
    if rank == 0 and not args.skip_batch:
        batched = batched_leg(B, torch, dev)
    if rank == 0 and not args.skip_learned:
        learned = learned_leg(args, B, torch, dev)

    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic",
        "config": dict(WORKLOAD, parallelism="replicas" if world > 1 else "single",
                       l2="flushed (256 MB write) before every timed solve; the 5.4 GB Krylov basis exceeds L2",
                       iterations=infos[-1]["iters"], outer=infos[-1]["outer"], relres=infos[-1]["relres"],
                       all_converged=ok, setup_ms=setup_ms),
        "error": error,
        "fp64": fp64,
        "e2e": {"value": 1000.0 / e2e_ms, "unit": UNIT, "h2d_bytes_per_step": N * 16, "d2h_bytes_per_step": N * 16,
                "path": "sg_gmres with host_io=1 (pinned host b and x copied inside the call)"},
        "gpu_launches": launches,
        "clocks": clocks,
        "tuning": tuning,
    }
    # the dominant kernel of the step by share of the solve's kernel time is
    # the tensor-core transform (28.8 % of the 511^2 solve with the binary16
    # basis, against 19.6 % for CGS2 pass 2, the largest HBM-bound kernel,
    # whose roofline is reported beside it)
    if top:
        line["roofline"] = top
    if cgs:
        line["roofline_cgs2"] = cgs
    if mv:
        line["matvec"] = mv
    if cfg2:
        line["cfg2_127"] = cfg2
    if cfg1:
        line["cfg1_1d"] = cfg1
    if batched:
        line["batched"] = batched
    if learned:
        line["learned"] = learned
    if world == 1 and not args.skip_cpu:
        S, M = oracle_sample_setup()
        n_sample = S.A.shape[0]
        steps511 = fp64["iterations"]
        per = [oracle_extrapolate(oracle_sample_step_seconds(S, M), n_sample, steps511) for _ in range(2)]
        line["cpu_baseline"] = {"value": 1.0 / statistics.mean(per), "unit": UNIT, "cores": os.cpu_count(),
                                "kind": "oracle", "sample": oracle_sample_text(n_sample, steps511, 2)}
        del S, M
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-matvec", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-learned", action="store_true")
    ap.add_argument("--skip-configs", action="store_true", help="skip the 127x127 and 1D legs")
    ap.add_argument("--quick", action="store_true", help="one FP64 solve instead of two")
    ap.add_argument("--learned-train", type=int, default=4096, help="training solves of the warm-start network")
    ap.add_argument("--learned-test", type=int, default=256, help="held-out solves of the warm-start leg")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
