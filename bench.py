#!/usr/bin/env python
"""Benchmark of the hybridised Crouzeix-Raviart solve on one GB300 per rank.

A step is one pass of the hot path over one synthetic problem: the coupled
element blocks (cr_assemble_coupled), the element-wise condensation into
G W = S (cr_hybridise), the Krylov solve to a relative residual of 1e-10
(cr_solve) and the element-wise recovery of U and P (cr_recover_up).  The
mesh topology (cr_mesh_load, host) is set up once and reported separately.

Metric: time to solution (seconds per step, lower is better), mixed precision
against FP64.  The default workload is the 3D transient Stokes problem on 64^3
cubes (1,572,864 Kuhn tetrahedra, 9.4 M unknowns, nu = 1, dt = 1e-3).  `value`
is the first solver of --precs (by default PCG in float-float with FP64
reliable updates and the Chebyshev polynomial preconditioner of degree 24, its
steps in FP32 on BF16 values of G); every timed solver (that one, its FP32-value
and float-float variants, float-float and native FP64 Jacobi-PCG, the FP64
Chebyshev PCG, float-float with BF16 low parts) is reported
under "precisions" with its roofline and its speed-up over FP64 Jacobi-PCG,
and the FP32 PCG inside FP64 refinement is attempted once with a bounded
iteration budget and its exit reported.  The 2D 512x512 workload follows
under "other_workloads".  Each timed step is bracketed by CUDA events on the
caller's stream; a 512 MB buffer is written between steps to flush L2.  A
step whose solve ends above the tolerance fails the run.

With --gpus N > 1 (torchrun), every rank solves its own replica of the
workload (the path has no exchange step: replicas only); the time is the
maximum over ranks.  `--impl reference` times the CPU FP64 oracle instead.
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

WORKLOADS = {
    "cfg1": "2D transient Stokes, 16x16 squares -> 512 triangles, nu=1, dt=1e-2, manufactured source",
    "cfg2": "2D transient Stokes, 512x512 squares -> 524,288 triangles perturbed +-0.2h, nu=1, dt=1e-3, "
            "8-mode Fourier source",
    "cfg3": "3D transient Stokes, 64^3 cubes -> 1,572,864 Kuhn tetrahedra, nu=1, dt=1e-3, Fourier source",
    "cfg4": "batch: 64 2D transient Stokes problems on n x n squares split into perturbed triangles, n log-uniform "
            "in [8, 256] (seed 2), 4 Fourier right-hand sides each, nu=1, dt=1e-3, one persistent batched PCG launch",
    "cfg5": "2D Navier-Stokes Newton step, 1024x1024 squares -> 2,097,152 triangles, Re=100, dt=1e-3, "
            "linearised about a seeded stream-function field",
}
METRIC = "time-to-solution at relative residual 1e-10 (hybridise + solve + recover)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg3", choices=sorted(WORKLOADS))
    ap.add_argument("--also", default=None,
                    help="comma-separated further workloads timed after the headline with their own default "
                         "solvers (default: cfg2 after cfg3; 'none' for none)")
    ap.add_argument("--steady", type=int, default=0,
                    help="cfg5: the steady (mu = 0) Newton step, solved by flexible GMRES on the coupled system "
                         "preconditioned by transient Stokes solves (mu_pre = --mu-pre)")
    ap.add_argument("--mu-pre", type=float, default=1.0, help="steady solves: mu of the preconditioning step")
    ap.add_argument("--mixed-attempt", type=int, default=1,
                    help="attempt FP32 PCG inside FP64 refinement once (bounded) and report its exit")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--poly-degree", type=int, default=0,
                    help="Chebyshev solvers: degree of the polynomial preconditioner (default 4)")
    ap.add_argument("--poly-ratio", type=float, default=0.0,
                    help="Chebyshev solvers: ratio of the interval's ends (default 1000 in 2D, 100 in 3D)")
    ap.add_argument("--graph", type=int, default=1, help="multi-kernel path: replay iteration chunks as graphs")
    ap.add_argument("--persistent", type=int, default=1, help="PCG in one cooperative persistent launch")
    ap.add_argument("--precs", default=None,
                    help="comma-separated solvers to time, the first is the headline (default: "
                         "ff_chebbf,ff_cheb32,ff_cheb,fp64_cheb,ff,fp64,ff_bf16 in 2D; "
                         "ff_chebbf,ff_cheb32,ff_cheb,ff,fp64,fp64_cheb,ff_bf16 for cfg3; ff_chebbf,ff for cfg5; ff for "
                         "cfg4)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--sample-iters", type=int, default=30)
    ap.add_argument("--sample-repeats", type=int, default=1, help=argparse.SUPPRESS)
    ap.add_argument("--check-every", type=int, default=16,
                    help="iterations per convergence check (persistent: x64 iterations per launch)")
    ap.add_argument("--deflate", type=int, default=0,
                    help="with --time-steps: also run the loop deflated by this many Ritz vectors, recorded by "
                         "the first step's solve over its first --lanczos iterations; with --steady: deflate the "
                         "inner solves by Ritz vectors of their G (--lanczos FP64 PCG steps)")
    ap.add_argument("--lanczos", type=int, default=200, help="PCG iterations that give the Ritz vectors (--deflate)")
    ap.add_argument("--time-steps", type=int, default=0,
                    help="also time this many implicit Euler steps of the transient workload")
    ap.add_argument("--compare-coupled", action="store_true",
                    help="also time the coupled system solved without hybridisation (MINRES)")
    ap.add_argument("--mesh-n", type=int, default=0,
                    help="profiling runs only: mesh size n in place of the workload's (n x n or n^3 cells)")
    ap.add_argument("--max-iter", type=int, default=0,
                    help="profiling runs only: stop every solve after this many iterations (no convergence check)")
    args = ap.parse_args()
    if args.precs is None:
        args.precs = default_precs(args.workload)
    args.precs = supported_precs(args.workload, args.precs, steady=bool(args.steady))
    if args.also is None:
        args.also = "cfg2" if args.workload == "cfg3" else ""
    args.also = [w for w in args.also.split(",") if w and w != "none" and w != args.workload]
    for w in args.also:
        if w not in WORKLOADS or w in ("cfg4", "cfg5"):
            ap.error(f"--also takes single-system Stokes workloads (cfg1, cfg2, cfg3), not {w}")
    return args


def default_precs(workload):
    """The fastest measured solver of each workload first: float-float PCG with the
    Chebyshev preconditioner whose steps run in FP32 on BF16 values of G (four times fewer
    CG iterations; the preconditioner's bytes cut to a third), then the same with FP32
    values and with float-float steps, float-float and FP64 Jacobi-PCG in the persistent
    kernel, the FP64 Chebyshev PCG (whose SpMV is bound by the FP64 pipe) and the
    BF16-low-part Jacobi variant."""
    if workload == "cfg3":
        return "ff_chebbf,ff_cheb32,ff_cheb,ff,fp64,fp64_cheb,ff_bf16"
    if workload == "cfg5":
        return "ff_chebbf,ff"   # each is a Newton step of several seconds
    return "ff_chebbf,ff_cheb32,ff_cheb,fp64_cheb,ff,fp64,ff_bf16"


def supported_precs(workload, precs, steady=False):
    """The Chebyshev-preconditioned PCG serves the single transient Stokes solve and the
    inner solves of the Newton steps (transient and steady); the batch keeps its
    Jacobi-preconditioned persistent kernel."""
    if workload == "cfg4":
        return ",".join(x for x in precs.split(",") if x and x not in CHEB_PRECS) or "ff"
    return precs


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def load_problem(name, n=None, steady=False):
    """Mesh, coefficients, sources and (for Navier-Stokes) the linearisation field;
    n (profiling runs only) replaces the workload's mesh size.  cfg5 is a transient
    Newton step (dt = 1e-3), or with `steady` the steady (mu = 0) one."""
    import numpy as np
    import synth
    p = synth.config_problem(name, n=n or None)
    if name == "cfg5":
        p["mu"] = 0.0 if steady else 1000.0
        p["conv"] = "newton"
    return p, np


PRECS = {
    # name: (cr_solve options, matrix value bytes, vector bytes, description)
    "fp64": (dict(prec="fp64", max_iter=200000), 8, 8, "Jacobi-PCG, native FP64"),
    "ff": (dict(prec="ff", max_iter=200000, inner_tol=0.01), 8, 8,
           "Jacobi-PCG in float-float (FP32 pairs, 48-bit significand) with FP64 reliable updates"),
    "ff_bf16": (dict(prec="ff_bf16", max_iter=200000, inner_tol=0.1), 6, 8,
                "Jacobi-PCG in float-float, G low plane in BF16 (6 B/value), FP64 reliable updates"),
    "mixed": (dict(prec="mixed", max_iter=400000, inner_tol=1e-4), 4, 4,
              "FP32 Jacobi-PCG restarted inside FP64 iterative refinement"),
    "fp64_cheb": (dict(prec="fp64", max_iter=200000, precond="chebyshev", poly_degree=4), 8, 8,
                  "PCG, native FP64, Chebyshev polynomial preconditioner of degree {degree} (Jacobi-preconditioned "
                  "Chebyshev steps under the Gershgorin bound; interval ratio {ratio}), graph-replayed kernels"),
    "ff_cheb": (dict(prec="ff", max_iter=200000, precond="chebyshev", poly_degree=4, inner_tol=0.01), 8, 8,
                "PCG in float-float (FP32 pairs) with FP64 reliable updates, Chebyshev polynomial preconditioner "
                "of degree {degree} (interval ratio {ratio}), graph-replayed kernels"),
    "ff_cheb32": (dict(prec="ff", max_iter=200000, precond="chebyshev", poly_degree=4, inner_tol=0.01,
                       poly_prec="fp32"), 4, 4,
                  "PCG in float-float (FP32 pairs) with FP64 reliable updates, Chebyshev polynomial preconditioner "
                  "of degree {degree} whose steps run in FP32 on the FP32 values of G (interval ratio {ratio}), "
                  "graph-replayed kernels"),
    "ff_chebbf": (dict(prec="ff", max_iter=200000, precond="chebyshev", poly_degree=4, inner_tol=0.01,
                       poly_prec="bf16"), 2, 4,
                  "PCG in float-float (FP32 pairs) with FP64 reliable updates, Chebyshev polynomial preconditioner "
                  "of degree {degree} whose steps run in FP32 on BF16 values of G (interval ratio {ratio}), "
                  "graph-replayed kernels"),
}
CHEB_PRECS = ("fp64_cheb", "ff_cheb", "ff_cheb32", "ff_chebbf")
# bytes per unknown that a Chebyshev step moves besides its SpMV: r read, d read and written,
# the Jacobi scale read
CHEB_EXTRA = {"fp64_cheb": 4 * 8, "ff_cheb": 3 * 8 + 4, "ff_cheb32": 8 + 2 * 4 + 4, "ff_chebbf": 8 + 2 * 4 + 4}

CHEB_RATIO = {2: 1000.0, 3: 100.0}
FP64_PEAK_TFLOPS = 1.25   # nominal GB300 FP64 rate (non-tensor)


# Chebyshev degree and interval ratio per dimension.  Steps in FP32 (on FP32 or BF16
# values) cost a fraction of a CG iteration's float-float SpMV, update and direction, so
# those solvers take a high degree (fewer CG iterations, more steps); measured on the
# 512^2 and 64^3 workloads: 2D degree 24 / ratio 10000 0.145 s against 0.256 s at degree
# 4 / ratio 1000, 3D degree 24 / ratio 3000 0.471 s against 0.666 s at degree 4 / ratio
# 100 (degrees 16 to 32 lie within 4% of these).  The float-float and FP64 steps cost as
# much as the CG iteration itself and stay at degree 4.
CHEB_DEGREE_FP32_STEPS = {2: 24, 3: 24}
CHEB_RATIO_FP32_STEPS = {2: 10000.0, 3: 3000.0}


def cheb_degree(args, prec, d):
    """Degree of the Chebyshev preconditioner of solver `prec` on a d-dimensional mesh."""
    if getattr(args, "poly_degree", 0):
        return args.poly_degree
    return CHEB_DEGREE_FP32_STEPS[d] if prec in ("ff_cheb32", "ff_chebbf") else PRECS[prec][0]["poly_degree"]


def cheb_ratio(args, prec, d):
    """Interval ratio of the Chebyshev preconditioner of solver `prec` (dimension d)."""
    if getattr(args, "poly_ratio", 0.0):
        return args.poly_ratio
    return CHEB_RATIO_FP32_STEPS[d] if prec in ("ff_cheb32", "ff_chebbf") else CHEB_RATIO[d]


def solver_text(args, prec, d):
    """The solver's description with the degree and ratio of this run."""
    text = PRECS[prec][3]
    if prec in CHEB_PRECS:
        text = text.format(degree=cheb_degree(args, prec, d), ratio=f"{cheb_ratio(args, prec, d):g}")
    return text


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant kernel of a
# solver, from one ncu capture: bytes per CG iteration (the persistent kernel) or per launch
# (the Chebyshev steps).  Each entry records the SHA-256 of the kernel's source (whole files,
# or the kernel's own section of a file between two marker lines) when it was captured; the
# bench reports it only while that source is unchanged, else null.
KERNEL_SOURCES = {
    "persist": ["persist.cu", "persist.h", "ff.cuh", "device_common.cuh"],
    "cheb_ff": [("solve.cu", "// Chebyshev step j: zout = zin + d_j, d_j = c1_j d + c2_j M^{-1} (r - G zin); on the",
                 "// p = z + beta p   (first: p = z)"), "ff.cuh", "device_common.cuh"],
    "cheb_rows1": [("solve.cu", "// Chebyshev step j in FP32 on the FP32 (or BF16) values of G; the last step forms",
                    "// ---- the FP32-step Chebyshev kernel, two rows per thread ----"), "ff.cuh", "device_common.cuh"],
    "cheb_rows2": [("solve.cu", "// ---- the FP32-step Chebyshev kernel, two rows per thread ----",
                    "// ---- the FP32-step Chebyshev kernel on slices staged in shared memory ----"),
                   "ff.cuh", "device_common.cuh"],
    "cheb_staged": [("solve.cu", "// ---- the FP32-step Chebyshev kernel on slices staged in shared memory ----",
                     "// Which form of the FP32 Chebyshev step runs"), "ff.cuh", "device_common.cuh"],
}
TRAFFIC = {
    # (workload, solver, kernel form or None): {"per": "iteration" | "launch", "bytes": B,
    # "sources": key, "sha256": digest}
    # the persistent float-float kernel on the 64^3 workload: two launches of 64 iterations,
    # 164.43 GB and 168.86 GB read + written
    ("cfg3", "ff", None): {"per": "iteration", "bytes": (164.431e9 + 168.859e9) / 2 / 64, "sources": "persist",
                           "sha256": "a5c561643bcd9514354b9d52efa8b149f579ce03c2e132758f392019507be00e"},
    # the FP32 Chebyshev step on BF16 values: three launches each on the 64^3 and 512^2
    # workloads, read + written
    ("cfg3", "ff_chebbf", "staged"): {
        "per": "launch", "bytes": (655521280 + 65956608 + 655623680 + 63242752 + 655530240 + 62977792) / 3,
        "sources": "cheb_staged", "sha256": "d34bb5e8d04d3b18ed131a58267950ba89cf11291a7f35ae2fbf9d1e046423b6"},
    ("cfg2", "ff_chebbf", "staged"): {
        "per": "launch", "bytes": (75430144 + 1292544 + 75429120 + 45824 + 75427328 + 56064) / 3,
        "sources": "cheb_staged", "sha256": "d34bb5e8d04d3b18ed131a58267950ba89cf11291a7f35ae2fbf9d1e046423b6"},
    # the persistent FP64 and FF_BF16 kernels on the 64^3 workload: two launches of 64 iterations each
    ("cfg3", "fp64", None): {"per": "iteration",
                             "bytes": (148678149120 + 19170485248 + 150336442112 + 19184686592) / 2 / 64,
                             "sources": "persist", "sha256": "a5c561643bcd9514354b9d52efa8b149f579ce03c2e132758f392019507be00e"},
    ("cfg3", "ff_bf16", None): {"per": "iteration",
                                "bytes": (123646610688 + 19144310272 + 127633991680 + 19611470080) / 2 / 64,
                                "sources": "persist", "sha256": "a5c561643bcd9514354b9d52efa8b149f579ce03c2e132758f392019507be00e"},
    # the FP32 Chebyshev step on FP32 values: two rows per thread on 64^3, one on 512^2
    ("cfg3", "ff_cheb32", "rows2"): {
        "per": "launch", "bytes": (1048752128 + 48134400 + 1048759296 + 44839168 + 1048767488 + 45010688) / 3,
        "sources": "cheb_rows2", "sha256": "f8ad74ed6aaa33a0b42db85c86ff8cd8f66766b3e52c5d1003ef7c1f609922b5"},
    ("cfg2", "ff_cheb32", "rows1"): {
        "per": "launch", "bytes": (106844416 + 2734848 + 106842880 + 111104 + 106854656 + 172544) / 3,
        "sources": "cheb_rows1", "sha256": "f5245097897897035a7bea13dfcd68e1200d7f1b200bb09776c9486c1f58276d"},
    # the float-float Chebyshev step (occupancy-sized grid)
    ("cfg3", "ff_cheb", None): {
        "per": "launch", "bytes": (1910210816 + 113576960 + 1910211328 + 109615616 + 1910217728 + 110364416) / 3,
        "sources": "cheb_ff", "sha256": "282b6805c17fe174f84a97c904a5c96d72d9b3226acd7b76783095ad5bcd0c72"},
    ("cfg2", "ff_cheb", None): {
        "per": "launch", "bytes": (182250496 + 4264960 + 182249216 + 2390784 + 182252032 + 1692928) / 3,
        "sources": "cheb_ff", "sha256": "282b6805c17fe174f84a97c904a5c96d72d9b3226acd7b76783095ad5bcd0c72"},
    ("cfg3", "ff_chebbf", "rows2"): {
        "per": "launch", "bytes": (655517184 + 47112448 + 655496704 + 44532736 + 655502592 + 44279296) / 3,
        "sources": "cheb_rows2", "sha256": "f8ad74ed6aaa33a0b42db85c86ff8cd8f66766b3e52c5d1003ef7c1f609922b5"},
    ("cfg2", "ff_chebbf", "rows2"): {
        "per": "launch", "bytes": (75431424 + 1131776 + 75428096 + 68864 + 75427840 + 38144) / 3,
        "sources": "cheb_rows2", "sha256": "f8ad74ed6aaa33a0b42db85c86ff8cd8f66766b3e52c5d1003ef7c1f609922b5"},
}


def sources_sha(key):
    """SHA-256 over the named sources of the CUDA library, in order: a file name stands for
    the whole file, (file, start, end) for its text from the start marker up to the end
    marker (None if a marker is missing)."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[key]:
        name = f if isinstance(f, str) else f[0]
        with open(os.path.join(ROOT, "paper_2101_03777_gb300", "csrc", name), "rb") as fh:
            data = fh.read()
        if not isinstance(f, str):
            i = data.find(f[1].encode())
            j = data.find(f[2].encode(), i + 1) if i >= 0 else -1
            if i < 0 or j < 0:
                return None
            data = data[i:j]
        h.update(data)
    return h.hexdigest()


def measured_traffic(workload, prec, form=None):
    """(bytes, per) from the capture table, or (None, reason) when there is no capture of
    this kernel build (form: the Chebyshev step kernel's form, for the FP32-step solvers)."""
    t = TRAFFIC.get((workload, prec, form))
    if not t:
        return None, "no ncu capture of this kernel on this workload"
    if sources_sha(t["sources"]) != t["sha256"]:
        return None, "the kernel's sources changed since the ncu capture"
    return t["bytes"], t["per"]


SPMV_KERNEL = {"fp64": "k_pcg_spmv<FP64>", "ff": "kf_spmv<float-float>", "ff_bf16": "kf_spmv<float+bf16>",
               "mixed": "k_pcg_spmv<FP32>", "fp64_cheb": "k_cheb_step<FP64> (SpMV + Chebyshev update)",
               "ff_cheb": "kf_cheb_step<float-float> (SpMV + Chebyshev update)",
               "ff_cheb32": "k32_cheb_step<float> (FP32 SpMV + Chebyshev update)",
               "ff_chebbf": "k32_cheb_step<bf16> (BF16-value SpMV + Chebyshev update)"}
DTYPE = {"fp64": "f64", "ff": "f32x2 (float-float)", "ff_bf16": "f32x2 (float-float; G low part bf16)",
         "mixed": "f32 (f64 refinement)", "fp64_cheb": "f64", "ff_cheb": "f32x2 (float-float)",
         "ff_cheb32": "f32x2 (float-float CG; f32 preconditioner steps)",
         "ff_chebbf": "f32x2 (float-float CG; f32 preconditioner steps on bf16 values)"}


def cheb_form(d, prec):
    """Form of the FP32 Chebyshev step kernel (rows1, rows2, staged) the library runs for
    solver `prec` on a d-dimensional mesh, or None for the other solvers."""
    pp = PRECS[prec][0].get("poly_prec")
    if pp not in ("fp32", "bf16"):
        return None
    from paper_2101_03777_gb300 import crhyb
    return crhyb.cr_chebyshev_step_form(d, pp)


def kernel_label(d, prec):
    """Name of the dominant kernel of solver `prec`, with the step kernel's form."""
    form = cheb_form(d, prec)
    if not form:
        return SPMV_KERNEL[prec]
    name = {"rows1": "k32_cheb_step", "rows2": "k32_cheb_step2", "staged": "k32_cheb_step_staged"}[form]
    return SPMV_KERNEL[prec].replace("k32_cheb_step", name, 1)


def solve_opts(prec, tol, graph, profile, persistent):
    o = dict(PRECS[prec][0])
    o.update(method="pcg", tol=tol, use_graph=graph, profile=profile, persistent=persistent)
    return o


def max_over_ranks(value, world, device="cuda"):
    """The largest of the ranks' values (each rank times its own replica; the job
    takes as long as the slowest).  world 1 returns the value unchanged."""
    if world <= 1:
        return float(value)
    import torch
    x = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(x, op=torch.distributed.ReduceOp.MAX)
    return float(x.item())


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle sample (run in a child process with one BLAS thread)
# ---------------------------------------------------------------------------
CPU_SAMPLE_N = {"cfg3": 32}   # workloads whose CPU sample runs on a coarser mesh of the same family


def cpu_model():
    """The host CPU's model name (lscpu), or the platform's processor string."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_sample(name, iters, repeats=1):
    """Time the oracle and extrapolate its time to solution on the workload.

    The set-up with hybridisation and the recovery are timed on the workload's
    mesh (for cfg3 on the 32^3 mesh of the same family, scaled by the element
    count, both being element-local), `iters` Jacobi-PCG iterations are timed on
    the same mesh (their cost scaled by the number of stored entries of G), and
    the PCG time is scaled to the oracle's own iteration count to a relative
    residual of 1e-10 on the full workload (oracle/iteration_counts.json).  With
    repeats > 1 the PCG sample and the recovery are timed that many times after
    one set-up ("values": one extrapolated time per repeat)."""
    import numpy as np
    import synth
    from oracle import hybrid, krylov, pipeline
    counts = json.load(open(os.path.join(ROOT, "oracle", "iteration_counts.json")))
    if name not in counts:
        raise RuntimeError(f"the CPU oracle sample covers the one-system Stokes PCG workloads {sorted(counts)}")
    full = counts[name]["pcg_iterations"]
    p = synth.config_problem(name, n=CPU_SAMPLE_N.get(name))
    t0 = time.perf_counter()
    topo, geom, A_K, D_K, R_K = pipeline.setup(p["coords"], p["elems"], p["nu"], p["mu"], p["fbar"][0], p["conv"])
    h = hybrid.hybridise(topo, A_K, D_K, R_K, p["mu"])
    t1 = time.perf_counter()
    runs = []
    for _ in range(max(repeats, 1)):
        ta = time.perf_counter()
        x, it, _ = krylov.pcg(h["G"], h["S"], krylov.jacobi(h["G"]), rtol=1e-30, maxit=iters)
        tb = time.perf_counter()
        hybrid.recover(h, topo, x)
        runs.append((tb - ta, time.perf_counter() - tb, it))
    t2 = t1 + runs[-1][0]
    t3 = t2 + runs[-1][1]
    it = runs[-1][2]
    ne_s, nnz_s = int(p["elems"].shape[0]), int(h["G"].nnz)
    # full-workload sizes: element count from the generator's definition, entries of G per row
    # are the same on the coarser mesh of the same family up to the boundary layer
    if name in CPU_SAMPLE_N:
        nf = int(CPU_SAMPLE_N[name])
        nF = 64
        el_scale = (nF / nf) ** 3
        nnz_scale = el_scale
        where = f"the {nf}^3 mesh of the same family ({ne_s} tetrahedra, scaled x{el_scale:.0f} to {nF}^3)"
    else:
        el_scale = nnz_scale = 1.0
        where = "the full mesh"
    per_it = (t2 - t1) / max(it, 1) * nnz_scale
    setup_s = (t1 - t0) * el_scale
    rec_s = (t3 - t2) * el_scale
    total = setup_s + per_it * full + rec_s
    per_repeat = [setup_s + pcg_s / max(k, 1) * nnz_scale * full + rec * el_scale for pcg_s, rec, k in runs]
    return {"value": total, "values": per_repeat, "unit": "s", "cores": 1, "kind": "oracle", "extrapolated": True,
            "sample": f"{name} on {where}: set-up + hybridise {t1 - t0:.2f} s, {it} Jacobi-PCG iterations "
                      f"({(t2 - t1) / max(it, 1) * 1e3:.1f} ms each, {per_it * 1e3:.1f} ms scaled), recover "
                      f"{t3 - t2:.2f} s; PCG scaled to the oracle's {full} iterations to 1e-10 on the full "
                      f"workload; numpy/scipy with 1 BLAS thread on a {os.cpu_count()}-core host "
                      f"({cpu_model()})",
            "measured_s": t3 - t0, "cpu_model": cpu_model(), "sample_elements": ne_s, "sample_nnz": nnz_s}


def run_cpu_sample_child(name, iters, repeats=1):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", name, "--sample-iters", str(iters),
                        "--sample-repeats", str(repeats)],
                       capture_output=True, text=True, env=env, timeout=1800)
    for line in r.stdout.splitlines()[::-1]:
        if line.startswith("{"):
            return json.loads(line)
    raise RuntimeError("CPU oracle sample failed: " + r.stderr[-2000:])


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def algorithmic_spmv_bytes(mesh_faces_elems, nf, d, vbytes, xbytes):
    """Bytes one SpMV must move: nnz*v + blocks*4 (int32 column) + N*(x + y)."""
    import numpy as np
    fe = mesh_faces_elems
    s = np.bincount(fe.ravel())
    blocks = int((s.astype(np.int64) ** 2).sum() - nf)     # sum_K s_K (s_K - 1) + F_int
    nnz = blocks * d * d
    N = nf * d
    return nnz * vbytes + blocks * 4 + N * 2 * xbytes, blocks, nnz


def check_step(st, tol, what):
    """A timed step counts only if its solve met the tolerance (FP64 true residual)."""
    if st["status"] != 0 or not (st["relres"] <= tol):
        raise RuntimeError(f"{what}: the solve ended with status {st['status']} at relative residual "
                           f"{st['relres']:.3e} > tol {tol:.1e}; the step is rejected")


def run_ours(args, rank, world, workload=None, precs=None, extras=True):
    """Time the solvers `precs` (the first is the headline) on `workload`."""
    import numpy as np
    import torch
    from paper_2101_03777_gb300 import build, crhyb

    workload = workload or args.workload
    precs = precs or [x for x in args.precs.split(",") if x]
    build.build_library()
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    p, _ = load_problem(workload, args.mesh_n, steady=bool(args.steady) and workload == "cfg5")
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_note = "of measured" if "hbm_gbs" in peaks else "of fallback"

    w_dev = None
    tm0 = time.perf_counter()
    mesh = crhyb.cr_mesh_load(p["coords"], p["elems"])
    mesh_load_s = time.perf_counter() - tm0
    if p["conv"] != "none":
        import synth
        xs = p["coords"][crhyb.cr_mesh_faces(mesh)].mean(axis=1)
        w_dev = torch.from_numpy(synth.stream_velocity(xs, seed=3)).cuda()
    d, nf, ne = mesh.dim, mesh.nf, mesh.ne
    n = nf * d
    fe, _ = crhyb.cr_mesh_face_elements(mesh)
    fbar_host = torch.from_numpy(p["fbar"]).pin_memory()
    fbar_dev = fbar_host.cuda()
    W = torch.zeros(n, dtype=torch.float64, device="cuda")
    U = torch.zeros(n, dtype=torch.float64, device="cuda")
    P = torch.zeros(ne, dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    newton = p["conv"] != "none"

    def step(prec, fb, Wt, Ut, Pt, profile=False, persistent=None, extra=None):
        persistent = args.persistent if persistent is None else persistent
        system = crhyb.cr_assemble_coupled(mesh, p["nu"], p["mu"], fb, conv=p["conv"], w=w_dev)
        if newton and p["mu"] == 0.0:
            # the steady Newton step: flexible GMRES on its coupled system, each step
            # preconditioned by a transient Stokes solve (SPD G, persistent PCG)
            pre = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, p["nu"], args.mu_pre, fb),
                                     keep_fp32=(prec == "ff_cheb32"), keep_bf16=(prec == "ff_chebbf"),
                                     keep_ff=(prec in ("ff", "ff_cheb", "ff_cheb32", "ff_chebbf")),
                                     keep_ff_bf16=(prec == "ff_bf16"))
            o = dict(tol=args.tol, prec=PRECS[prec][0]["prec"], profile=profile, check_every=args.check_every,
                     restart=60)
            if prec in CHEB_PRECS:
                o.update(precond="chebyshev", poly_degree=cheb_degree(args, prec, d),
                         poly_ratio=cheb_ratio(args, prec, d), poly_prec=PRECS[prec][0].get("poly_prec", "same"))
            if args.max_iter:
                o["max_iter"] = args.max_iter
            if args.deflate and prec in CHEB_PRECS:
                # every inner solve shares G_mu: Ritz vectors of pre deflate them all (their Lanczos
                # run is part of the step)
                lo = {key: o[key] for key in ("precond", "poly_degree", "poly_ratio")}
                o["deflation"] = crhyb.cr_deflation_lanczos(pre, args.lanczos, args.deflate, **lo)[0]
            # the steady solve writes device arrays: the end-to-end run copies them to its host buffers
            Ud = Ut if Ut.is_cuda else torch.zeros(Ut.shape, dtype=torch.float64, device="cuda")
            Pd = Pt if Pt.is_cuda else torch.zeros(Pt.shape, dtype=torch.float64, device="cuda")
            st = crhyb.cr_solve_steady(system, pre, Ud, Pd, raise_on_error=not args.max_iter, **o)
            if not Ut.is_cuda:
                Ut.copy_(Ud)
                Pt.copy_(Pd)
            return st
        if newton:
            # the nonsymmetric Newton system (FP64 values for the outer GMRES) and the transient
            # Stokes system on the same mesh, whose PCG solves precondition it
            hyb = crhyb.cr_hybridise(system, keep_fp32=False)
            pre = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, p["nu"], p["mu"], fb),
                                     keep_fp32=(prec == "ff_cheb32"), keep_bf16=(prec == "ff_chebbf"),
                                     keep_ff=(prec in ("ff", "ff_cheb", "ff_cheb32", "ff_chebbf")),
                                     keep_ff_bf16=(prec == "ff_bf16"))
            o = dict(tol=args.tol, prec=PRECS[prec][0]["prec"], profile=profile, check_every=args.check_every)
            if prec in CHEB_PRECS:
                # the inner PCG with the Chebyshev preconditioner (multi-kernel, graph-replayed)
                o.update(precond="chebyshev", poly_degree=cheb_degree(args, prec, d),
                         poly_ratio=cheb_ratio(args, prec, d), poly_prec=PRECS[prec][0].get("poly_prec", "same"))
            if args.max_iter:
                o["max_iter"] = args.max_iter
            st = crhyb.cr_solve_preconditioned(hyb, pre, Wt, raise_on_error=not args.max_iter, **o)
            crhyb.cr_recover_up(hyb, Wt, Ut, Pt, normalise_p=True)
            return st
        hyb = crhyb.cr_hybridise(system, keep_fp32=(prec in ("mixed", "ff_cheb32")), keep_bf16=(prec == "ff_chebbf"),
                                 keep_ff=(prec in ("ff", "ff_cheb", "ff_cheb32", "ff_chebbf")),
                                 keep_ff_bf16=(prec == "ff_bf16"))
        o = solve_opts(prec, args.tol, args.graph and not profile, profile, persistent)
        o["check_every"] = args.check_every
        if o.get("precond") == "chebyshev":
            o["poly_ratio"] = cheb_ratio(args, prec, d)
            o["poly_degree"] = cheb_degree(args, prec, d)
        if args.max_iter:
            o["max_iter"] = args.max_iter
        if extra:
            o.update(extra)
        st = crhyb.cr_solve(hyb, Wt, raise_on_error=not args.max_iter and not extra, **o)
        crhyb.cr_recover_up(hyb, Wt, Ut, Pt, normalise_p=True)
        return st

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(prec, profile):
        for _ in range(args.warmup):
            step(prec, fbar_dev, W, U, P)
        torch.cuda.synchronize()
        times, stats = [], []
        for _ in range(args.steps):
            flush.fill_(1.0)
            barrier()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = step(prec, fbar_dev, W, U, P, profile)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            times.append(e0.elapsed_time(e1) / 1e3)
            stats.append(st)
            if not args.max_iter:
                check_step(st, args.tol, f"{workload} {prec}")
        return times, stats

    head = precs[0]
    clocks = ClockSampler(dev)
    clocks.start()
    runs = {prec: timed(prec, False) for prec in precs}
    clk = clocks.stop()
    # kernel timing (outside the timed steps): one step with CUDA events around every launch of the
    # dominant kernel, and one step of the multi-kernel path for the stand-alone SpMV
    prof = {}
    for prec in precs:
        flush.fill_(1.0)
        torch.cuda.synchronize()
        st_main = step(prec, fbar_dev, W, U, P, profile=True)
        st_spmv = None
        if not newton:
            flush.fill_(1.0)
            torch.cuda.synchronize()
            st_spmv = step(prec, fbar_dev, W, U, P, profile=True, persistent=0)
        prof[prec] = (st_main, st_spmv)

    # FP32 PCG inside FP64 iterative refinement, attempted once with a bounded budget
    mixed = None
    if extras and args.mixed_attempt and not newton and not args.max_iter:
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stm = step("mixed", fbar_dev, W, U, P, persistent=0, extra=dict(max_iter=40000, max_outer=60))
        torch.cuda.synchronize()
        mixed = {"solver": PRECS["mixed"][3], "status": stm["status_name"], "exit": stm.get("error", "converged"),
                 "relres": stm["relres"],
                 "inner_iterations": stm["iterations"], "refinement_steps": stm["outer"],
                 "seconds": time.perf_counter() - t0, "budget": "40,000 inner iterations, 60 refinement steps"}

    # end-to-end through the C-ABI with host buffers: pinned fbar in, U and P out to pinned host memory
    Uh = torch.empty(n, dtype=torch.float64).pin_memory()
    Ph = torch.empty(ne, dtype=torch.float64).pin_memory()
    Wh = torch.zeros(n, dtype=torch.float64).pin_memory()
    e2e = []
    for k in range(args.warmup + args.steps):
        flush.fill_(1.0)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = step(head, fbar_host, Wh, Uh, Ph)
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e.append(time.perf_counter() - t0)
            if not args.max_iter:
                check_step(st, args.tol, f"{workload} {head} (end to end)")

    def agg(v):
        return max_over_ranks(v, world)

    N = n

    def summary(prec):
        times, stats = runs[prec]
        tts = agg(statistics.mean(times))
        vb, xb = PRECS[prec][1], PRECS[prec][2]
        spmv_bytes, blocks, nnz = algorithmic_spmv_bytes(fe, nf, d, vb, xb)
        st_main, st_spmv = prof[prec]
        solver = solver_text(args, prec, d)
        spmv = None
        if st_spmv is not None and prec in CHEB_PRECS:
            # the Chebyshev steps: degree - 1 launches per CG iteration, each the SpMV over G fused
            # with the vector update (reads r, d, M^{-1}; writes d and the other z buffer)
            deg = cheb_degree(args, prec, d)
            step_bytes = spmv_bytes + CHEB_EXTRA[prec] * N
            nit = max(st_spmv["spmv_launches"], 1)
            ms = st_spmv["spmv_ms"] / (nit * (deg - 1))
            form = cheb_form(d, prec)
            tb, tnote = measured_traffic(workload, prec, form)
            spmv = {"kernel": kernel_label(d, prec), "bound": "hbm", "achieved": step_bytes / (ms * 1e-3) / 1e9,
                    "peak": hbm_peak, "unit": "GB/s", "frac": step_bytes / (ms * 1e-3) / 1e9 / hbm_peak,
                    "traffic": tb, "bytes_per_launch": step_bytes, "avg_launch_ms": ms,
                    "launches_timed": nit * (deg - 1), "peak_note": peak_note}
            if form:
                spmv["form"] = form
            if tb is None:
                spmv["traffic_note"] = tnote
        elif st_spmv is not None:
            # stand-alone SpMV launches of the multi-kernel path
            nl = max(st_spmv["spmv_launches"], 1)
            ms = st_spmv["spmv_ms"] / nl
            spmv = {"kernel": SPMV_KERNEL[prec], "bound": "hbm", "achieved": spmv_bytes / (ms * 1e-3) / 1e9,
                    "peak": hbm_peak, "unit": "GB/s", "frac": spmv_bytes / (ms * 1e-3) / 1e9 / hbm_peak,
                    "bytes_per_launch": spmv_bytes, "avg_launch_ms": ms, "launches_timed": nl,
                    "peak_note": peak_note}
        if newton and prec in CHEB_PRECS:
            # steady step with Chebyshev inner solves: the Chebyshev steps of the inner PCG dominate
            deg = cheb_degree(args, prec, d)
            step_bytes = spmv_bytes + CHEB_EXTRA[prec] * N
            nl = max(st_main["spmv_launches"], 1) * (deg - 1)
            ms = st_main["spmv_ms"] / nl
            roof = {"kernel": kernel_label(d, prec) + " (inner Stokes solves)", "bound": "hbm",
                    "achieved": step_bytes / (ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "frac": step_bytes / (ms * 1e-3) / 1e9 / hbm_peak, "traffic": None,
                    "bytes_per_launch": step_bytes, "avg_launch_ms": ms, "launches_timed": nl,
                    "peak_note": peak_note}
            if p["mu"] == 0.0:
                solver = ("steady Newton step: flexible GMRES(60) in FP64 on the coupled system (Eq. 10, mu = 0), "
                          f"each step preconditioned by one transient Stokes step (mu = {args.mu_pre:g}) of the "
                          f"hybrid method, inner {solver} to 1e-6")
            else:
                solver = ("Newton step: flexible GMRES(30) in FP64 on the nonsymmetric G, each step preconditioned "
                          f"by a solve with the transient Stokes G of the same mesh, inner {solver} to 0.1")
        elif newton:
            # the inner persistent PCG on the Stokes G (same mesh, same sliced ELL) dominates the step
            mb = 4 if prec != "fp64" else 8
            it_bytes = spmv_bytes + 9 * N * xb + 2 * N * mb
            piters = max(st_main["spmv_launches"], 1)
            kms = st_main["spmv_ms"]
            ach = it_bytes * piters / (kms * 1e-3) / 1e9
            roof = {"kernel": f"k_pcg_persist<{PRECS[prec][0]['prec']}> (inner Stokes PCG: SpMV + update + "
                              "direction phases)", "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                    "frac": ach / hbm_peak, "traffic": None, "bytes_per_iteration": it_bytes,
                    "iterations_timed": piters, "kernel_ms": kms, "peak_note": peak_note}
            if p["mu"] == 0.0:
                solver = ("steady Newton step: flexible GMRES(60) in FP64 on the coupled system (Eq. 10, mu = 0), "
                          f"each step preconditioned by one transient Stokes step (mu = {args.mu_pre:g}) of the hybrid "
                          f"method, inner {solver} to 1e-6")
            else:
                solver = ("flexible GMRES(30) in FP64 on the Newton system, each step preconditioned by an inner "
                          f"{solver} on the transient Stokes G of the same mesh to relative residual 0.1")
        elif prec in CHEB_PRECS:
            roof = dict(spmv)
        elif args.persistent:
            # the persistent PCG kernel: per iteration the SpMV plus the vector phases (the update
            # reads x, r, p, q and writes x, r; the direction reads r, p and writes p: 9 vector
            # passes) and the preconditioner read twice
            mb = 4 if prec != "fp64" else 8
            it_bytes = spmv_bytes + 9 * N * xb + 2 * N * mb
            piters = max(st_main["spmv_launches"], 1)
            kms = st_main["spmv_ms"]
            ach = it_bytes * piters / (kms * 1e-3) / 1e9
            nlaunch = max(st_main["kernel_launches"] - 1, 1)
            tb, tnote = measured_traffic(workload, prec)
            roof = {"kernel": f"k_pcg_persist<{PRECS[prec][0]['prec']}> (SpMV + update + direction phases)",
                    "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                    "traffic": tb * piters / nlaunch if tb is not None else None, "bytes_per_iteration": it_bytes,
                    "iterations_timed": piters, "bytes_per_launch": it_bytes * piters / nlaunch,
                    "avg_launch_ms": kms / nlaunch, "peak_note": peak_note}
            if tb is None:
                roof["traffic_note"] = tnote
            else:
                roof["traffic_per_iteration"] = tb
            if prec == "fp64":
                # the FP64 pipe: 2 flops per matrix entry and about 14 per unknown in the vector
                # phases (update, dots, direction), against the nominal FP64 rate (no measured peak)
                flops = 2 * nnz + 14 * N
                fl = flops * piters / (kms * 1e-3) / 1e12
                roof["alu"] = {"bound": "fp64", "achieved": fl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                               "frac": fl / FP64_PEAK_TFLOPS, "flops_per_iteration": flops,
                               "peak_note": "nominal FP64 rate; no measured FP64 peak"}
        else:
            roof = dict(spmv, traffic=None)
        return tts, {
            "value": tts, "unit": "s", "solver": solver, "iterations": stats[-1]["iterations"],
            "outer": stats[-1]["outer"], "relres": stats[-1]["relres"],
            "kernel_launches_per_step": int(statistics.mean(s["kernel_launches"] for s in stats)) + 4,
            "roofline": roof, "spmv": spmv}

    sums = {prec: summary(prec) for prec in precs}
    if "fp64" in sums:
        for prec in precs:
            sums[prec][1]["speedup_vs_fp64"] = sums["fp64"][0] / sums[prec][0]
    tts, hs = sums[head]
    tts_e2e = agg(statistics.mean(e2e))
    out = {
        "metric": METRIC, "value": tts, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tts * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[head], "data": "synthetic (seeded generators in synth/)",
        "config": {"workload": f"{workload}: {WORKLOADS[workload]}" + (" (steady, mu = 0)" if p["mu"] == 0.0 else ""),
                   "nf_int": nf, "unknowns": n,
                   "elements": ne, "solver": hs["solver"], "tol": args.tol, "iterations": hs["iterations"],
                   "outer": hs["outer"], "relres": hs["relres"], "mesh_load_s": mesh_load_s,
                   "l2": "512 MB flush between steps",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU", "graph": bool(args.graph),
                   "persistent": bool(args.persistent)},
        "roofline": hs["roofline"],
        "e2e": {"value": tts_e2e, "unit": "s", "h2d_bytes_per_step": int(p["fbar"].nbytes),
                "d2h_bytes_per_step": int(8 * (n + ne))},
        "gpu_launches": hs["kernel_launches_per_step"],
        "clocks": clk,
        "precisions": {prec: sums[prec][1] for prec in precs},
    }
    if "fp64" in sums and head != "fp64":
        out["speedup_vs_fp64"] = sums["fp64"][0] / tts
    if mixed is not None:
        out["mixed_fp32_refinement"] = mixed
    if extras and args.time_steps and not newton:
        # implicit Euler steps of the transient workload (mu = 1/dt) from rest: each step hands
        # U^n to the next right-hand side, hybridises, solves from the previous W (warm start)
        # and recovers U^{n+1}; timed as one region with CUDA events.  With --deflate the loop
        # runs again, deflated after its first step by Ritz vectors of that step's system
        # (their Lanczos run inside the timed region)
        prec = head
        o = solve_opts(prec, args.tol, args.graph, False, args.persistent)
        o["check_every"] = args.check_every
        if o.get("precond") == "chebyshev":
            o["poly_ratio"] = cheb_ratio(args, prec, d)
            o["poly_degree"] = cheb_degree(args, prec, d)

        def time_loop(k_defl):
            system = crhyb.cr_assemble_coupled(mesh, p["nu"], p["mu"], fbar_dev)
            Ut = torch.zeros(n, dtype=torch.float64, device="cuda")
            Wt = torch.zeros(n, dtype=torch.float64, device="cuda")
            iters, defl = [], []

            def time_step(k):
                crhyb.cr_system_set_previous(system, Ut)
                hyb = crhyb.cr_hybridise(system, keep_fp32=(prec in ("mixed", "ff_cheb32")),
                                         keep_bf16=(prec == "ff_chebbf"),
                                         keep_ff=(prec in ("ff", "ff_cheb", "ff_cheb32", "ff_chebbf")),
                                         keep_ff_bf16=(prec == "ff_bf16"))
                if k_defl and not defl:
                    # the first solve records its iterations and returns the Ritz vectors
                    st, dsp, _ = crhyb.cr_solve_ritz(hyb, Wt, args.lanczos, k_defl, use_x0=k > 0, **o)
                    defl.append(dsp)
                else:
                    st = crhyb.cr_solve(hyb, Wt, use_x0=k > 0, deflation=defl[0] if defl else None, **o)
                crhyb.cr_recover_up(hyb, Wt, Ut, P, normalise_p=True)
                iters.append(st["iterations"])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(args.time_steps):
                time_step(k)
            e1.record(stream)
            torch.cuda.synchronize()
            return agg(e0.elapsed_time(e1) / 1e3), iters, (defl[0].k if defl else 0)

        tl, iters, _ = time_loop(0)
        out["time_loop"] = {"steps": args.time_steps, "value": tl / args.time_steps, "unit": "s per step",
                            "precision": prec, "iterations_per_step": iters,
                            "note": "implicit Euler from rest, dt = 1/mu; each step warm-starts from the previous W"}
        if args.deflate:
            tld, iters_d, kept = time_loop(args.deflate)
            out["time_loop_deflated"] = {
                "steps": args.time_steps, "value": tld / args.time_steps, "unit": "s per step", "precision": prec,
                "iterations_per_step": iters_d, "vectors": kept, "lanczos_steps": args.lanczos,
                "speedup": tl / tld,
                "note": "the same loop; the first step's solve records its first iterations (cr_solve_ritz) and "
                        "their Ritz vectors deflate the solves of the later steps"}
    if extras and args.compare_coupled and not newton:
        # the paper's comparison: the same coupled system solved without hybridisation
        # (assembly + preconditioned MINRES to the same relative residual), one warm-up and
        # one timed step, outside the timed region of the headline
        def coupled_step():
            system = crhyb.cr_assemble_coupled(mesh, p["nu"], p["mu"], fbar_dev)
            cpl = crhyb.cr_coupled_create(system)
            return crhyb.cr_solve_coupled(cpl, U, P, tol=args.tol, prec="fp64", check_every=64)
        coupled_step()
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stc = coupled_step()
        e1.record(stream)
        torch.cuda.synchronize()
        tc = agg(e0.elapsed_time(e1) / 1e3)
        out["non_hybrid"] = {"solver": "preconditioned MINRES (FP64) on the coupled system of Eq. 10, diagonal "
                                       "velocity / Schur-diagonal pressure preconditioner",
                             "value": tc, "unit": "s", "iterations": stc["iterations"], "relres": stc["relres"],
                             "hybrid_speedup": tc / tts}
    return out


def run_batch(args, rank, world):
    """cfg4: every step hybridises the 64 problems, solves their 256 (problem, rhs)
    pairs in one batched persistent PCG and recovers U and P of every pair."""
    import numpy as np
    import torch
    import synth
    from paper_2101_03777_gb300 import build, crhyb

    build.build_library()
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_note = "of measured" if "hbm_gbs" in peaks else "of fallback"
    prec = [x for x in args.precs.split(",") if x][0]
    probs = synth.batch_problems(count=64, nrhs=4, lo=8, hi=256, seed=2)
    meshes = [crhyb.cr_mesh_load(q["coords"], q["elems"]) for q in probs]
    fb_host = [torch.from_numpy(q["fbar"]).pin_memory() for q in probs]
    fb_dev = [f.cuda() for f in fb_host]
    ns = [m.nf * m.dim for m in meshes]
    Ws = [torch.zeros(4 * n, dtype=torch.float64, device="cuda") for n in ns]
    Us = [torch.zeros(n, dtype=torch.float64, device="cuda") for n in ns]
    Ps = [torch.zeros(m.ne, dtype=torch.float64, device="cuda") for m in meshes]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    keep = dict(keep_fp32=False, keep_ff=(prec == "ff"), keep_ff_bf16=(prec == "ff_bf16"))
    tuned = {"bps": 0, "grouping": 0}

    def step(fbs, profile=False, outs=None):
        hybs = [crhyb.cr_hybridise(crhyb.cr_assemble_coupled(m, q["nu"], q["mu"], f), **keep)
                for m, q, f in zip(meshes, probs, fbs)]
        batch = crhyb.cr_batch_create(hybs, prec=prec, autotune=tuned["bps"] == 0, blocks_per_sm=tuned["bps"],
                                      rhs_grouping=tuned["grouping"])
        st = crhyb.cr_solve_batched(batch, Ws, tol=args.tol, max_iter=200000, profile=profile)
        if tuned["bps"] == 0:
            # later steps plan the batch with the autotuner's choice: its resident blocks per SM
            # and its grouping of the right-hand sides, read back from the number of systems
            info = batch.info()
            tuned["bps"] = info["blocks_per_sm"]
            tuned["grouping"] = {len(probs): 1, 4 * len(probs): 2}.get(info["nsys"], 3)
        for k, (h, W) in enumerate(zip(hybs, Ws)):
            for r in range(4):
                if outs is None:   # device U and P
                    crhyb.cr_recover_up(h, W[r * h.n:(r + 1) * h.n], Us[k], Ps[k], rhs=r)
                else:              # every pair's U and P into pinned host memory
                    Uh, Ph = outs
                    crhyb.cr_recover_up(h, W[r * h.n:(r + 1) * h.n], Uh[k][r * h.n:(r + 1) * h.n],
                                        Ph[k][r * h.mesh.ne:(r + 1) * h.mesh.ne], rhs=r)
        return st, batch.info()

    for _ in range(args.warmup):
        step(fb_dev)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    times, stats = [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, info = step(fb_dev)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        stats.append(st)
    clk = clocks.stop()
    flush.fill_(1.0)
    torch.cuda.synchronize()
    stp, info = step(fb_dev, profile=True)
    tts = statistics.mean(times)
    st = stats[-1]
    # end to end through the C-ABI with host buffers: pinned fbar in, U and P of all 256 pairs out
    Uh = [torch.empty(4 * n, dtype=torch.float64).pin_memory() for n in ns]
    Ph = [torch.empty(4 * m.ne, dtype=torch.float64).pin_memory() for m in meshes]
    e2e = []
    for k in range(args.warmup + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(fb_host, outs=(Uh, Ph))
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e.append(time.perf_counter() - t0)
    h2d = sum(int(q["fbar"].nbytes) for q in probs)
    d2h = sum(8 * 4 * (n + m.ne) for n, m in zip(ns, meshes))
    # algorithmic bytes of one batched iteration (all pairs active): per problem the SpMM over
    # G (values once for its 4 right-hand sides) plus the vector passes of 4 right-hand sides
    vb = {"ff": 8, "ff_bf16": 6, "fp64": 8}[prec]
    mb = 8 if prec == "fp64" else 4
    iters = [s["iterations"] for s in st]
    # the kernel runs every pair until its own convergence: weight each problem's bytes by its
    # mean iteration count over the timed persistent launches
    kms = stp[0]["spmv_ms"]
    work = 0.0
    j = 0
    for m in meshes:
        fe, _ = crhyb.cr_mesh_face_elements(m)
        sp, blocks, nnz = algorithmic_spmv_bytes(fe, m.nf, m.dim, vb, 8)
        N = m.nf * m.dim
        its = [stp[j + r]["iterations"] for r in range(4)]
        j += 4
        work += max(its) * (nnz * vb + blocks * 4) + sum(its) * (11 * N * 8 + 2 * N * mb)
    ach = work / (kms * 1e-3) / 1e9
    return {
        "metric": METRIC, "value": tts, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tts * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[prec], "data": "synthetic (seeded generators in synth/)",
        "config": {"workload": f"cfg4: {WORKLOADS['cfg4']}", "problems": len(probs), "pairs": len(st),
                   "unknowns_total": int(sum(ns)), "n_range": [min(q["n"] for q in probs), max(q["n"] for q in probs)],
                   "solver": PRECS[prec][3] + ", batched persistent launch", "tol": args.tol,
                   "iterations_min_max": [min(iters), max(iters)], "relres_max": max(s["relres"] for s in st),
                   "tiles": info["ntiles"], "grid": info["grid"], "blocks_per_sm_autotuned": info["blocks_per_sm"],
                   "rhs_per_system_autotuned": {1: 4, 2: 1, 3: 2}[tuned["grouping"]],
                   "l2": "512 MB flush between steps", "parallelism": "1 GPU"},
        "roofline": {"kernel": f"k_pcg_persist<{prec}, {({1: 4, 2: 1, 3: 2}[tuned['grouping']])} rhs> "
                                "(batched SpMM + update + direction phases)",
                     "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                     "traffic": None, "bytes_timed": work, "kernel_ms": kms, "peak_note": peak_note},
        "e2e": {"value": statistics.mean(e2e), "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(st[0]["kernel_launches"]) + 64 * 2 + 256 * 2,
        "clocks": clk,
    }


def run_reference(args, rank, world):
    """The CPU FP64 oracle as it stands, on the host cores (rank 0 only): one child
    process with one BLAS thread sets the sample mesh up once, then times W + K
    samples (Jacobi-PCG iterations and the recovery), each extrapolated to the
    workload's time to solution as cpu_sample describes."""
    if rank != 0:
        return None
    if args.workload not in ("cfg1", "cfg2", "cfg3"):
        return {"impl": "reference", "unavailable": f"the CPU oracle arm covers the one-system Stokes workloads "
                                                    f"(cfg1-cfg3), not {args.workload}"}
    info = run_cpu_sample_child(args.workload, args.sample_iters, repeats=args.warmup + args.steps)
    vals = info["values"][args.warmup:]
    v = statistics.mean(vals)
    cb = {k: info[k] for k in ("unit", "cores", "kind", "sample", "extrapolated", "cpu_model")}
    cb["value"] = v
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generators in synth/)",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}",
                       "solver": "Jacobi-PCG FP64 (CPU oracle, extrapolated from a bounded sample)",
                       "tol": args.tol},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.cpu_sample:
        print(json.dumps(cpu_sample(args.cpu_sample, args.sample_iters, args.sample_repeats)))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out:
            print(json.dumps(out))
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    out = run_batch(args, rank, world) if args.workload == "cfg4" else run_ours(args, rank, world)
    if args.also and not args.mesh_n:
        # further workloads, each with its own two fastest solvers, after the headline
        import gc
        import torch
        gc.collect()
        torch.cuda.empty_cache()
        out["other_workloads"] = {}
        for w in args.also:
            o = run_ours(args, rank, world, workload=w, precs=default_precs(w).split(",")[:2], extras=False)
            out["other_workloads"][w] = {k: o[k] for k in ("value", "unit", "dtype", "config", "roofline", "e2e",
                                                           "gpu_launches", "clocks", "precisions")}
            gc.collect()
            torch.cuda.empty_cache()
    if rank == 0:
        if args.mesh_n:
            out["config"]["mesh_n"] = args.mesh_n   # a profiling size, not the workload's
        if world == 1 and not args.no_cpu_baseline and not args.mesh_n:
            try:
                out["cpu_baseline"] = run_cpu_sample_child(args.workload, args.sample_iters)
            except Exception as e:  # reported, not fatal
                out["cpu_baseline"] = {"error": str(e)[:300]}
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
