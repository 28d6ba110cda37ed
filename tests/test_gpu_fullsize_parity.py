"""Element-wise U/P parity on meshes large enough to take the full-size code paths.

The smaller parity meshes (test_gpu_parity, test_gpu_chebyshev, test_gpu_batch)
fit in one pass of every kernel.  These meshes do not:
  * 2D 384 x 384 perturbed squares (cfg2 family): 441,600 face rows, more than
    the 311,296 rows (8 blocks of 256 threads on each of 152 SMs) at which the
    grid-stride loops of the three-kernel, Chebyshev and GMRES kernels start a
    second pass, and 1,725 tiles, more than the persistent kernel's resident
    blocks, so each block sweeps several tiles per phase;
  * 3D 32^3 Kuhn cubes (cfg3 family): 387,072 face rows, 1,512 tiles;
  * the batched workload itself (64 meshes, n from 9 to 234, 4 right-hand sides
    each, float-float, autotuned), whose largest problem runs alone on
    rebalanced tiles at the end of the solve;
  * a transient Newton step on 384 x 384 squares (flexible GMRES with inner
    float-float PCG);
  * the three forms of the FP32 Chebyshev step kernel (one row per thread,
    two rows per thread, slices staged in shared memory by bulk copies), each
    in a child process (CRHYB_CHEB_KERNEL fixes the form per process), on
    both meshes: more slices than resident blocks, so every block of the
    staged form sweeps several slices and flips its mbarrier phase.
The GPU solves to a relative residual of 1e-11 and recovers U and P (P
normalised to zero mean, Section 2 item 5); they must match the oracle's
within 1e-9 relative L2 (FP64, float-float, Chebyshev) or 1e-8 (float-float
with BF16 low parts), the tolerances of the parity tests.  The oracle's
truths (fullsize_truth.py) are computed in spawned worker processes while the
GPU solves run.  1e-11 is near the attainable accuracy at these sizes: the
oracle's own sparse LU of G leaves a relative residual of 1.6e-13 at 384 x 384,
and the GPU's FP64 PCG, whose true residual is evaluated in FP64, stagnates
between 1e-12 and 1e-11 there; on the oracle at 128 x 128 a PCG solve to 1e-13
recovers U within 1.5e-13 of the direct solve (the recovered U is far better
conditioned than W), so the U and P errors of a solve to 1e-11 stay orders of
magnitude below the tolerances.
"""

import multiprocessing
import os
import subprocess
import sys
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

import bench
import fullsize_truth as truth
import synth
from paper_2101_03777_gb300 import crhyb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N2D, N3D, NNEWTON = 384, 32, 384


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _largest_batch_problem():
    return int(np.argmax(synth.batch_sizes(64, 8, 256, 2)))


@pytest.fixture(scope="module")
def truths():
    """Futures of the oracle truths, started before the first GPU call of this module."""
    ex = ProcessPoolExecutor(max_workers=4, mp_context=multiprocessing.get_context("spawn"))
    k = _largest_batch_problem()
    fut = {
        "3d": ex.submit(truth.stokes_3d, N3D, 1e-12),
        "2d": ex.submit(truth.stokes_2d, N2D),
        "newton": ex.submit(truth.newton_2d, NNEWTON),
        "batch": ex.submit(truth.batch_problem, k),
        "batch_small": ex.submit(truth.batch_problem, int(np.argmin(synth.batch_sizes(64, 8, 256, 2)))),
    }
    yield fut
    ex.shutdown(wait=True, cancel_futures=True)


_GPU = {}


def gpu_problem(name):
    """Mesh and hybridised system (all value precisions kept) of a 2D or 3D case, cached."""
    if name not in _GPU:
        _GPU.clear()
        p = synth.config_problem("cfg2" if name == "2d" else "cfg3", n=N2D if name == "2d" else N3D)
        mesh = crhyb.cr_mesh_load(p["coords"], p["elems"])
        fb = torch.from_numpy(p["fbar"]).cuda()
        hyb = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, p["nu"], p["mu"], fb), keep_fp32=True,
                                 keep_bf16=True, keep_ff=True, keep_ff_bf16=True)
        _GPU[name] = (mesh, hyb)
    return _GPU[name]


def solve_recover(hyb, rhs=0, solver=None, **opts):
    n, ne = hyb.n, hyb.mesh.ne
    W = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = solver(W) if solver else crhyb.cr_solve(hyb, W, rhs=rhs, **opts)
    U = torch.zeros(n, dtype=torch.float64, device="cuda")
    P = torch.zeros(ne, dtype=torch.float64, device="cuda")
    crhyb.cr_recover_up(hyb, W, U, P, rhs=rhs, normalise_p=True)
    return st, U.cpu().numpy(), P.cpu().numpy()


SOLVERS = {
    "fp64-persistent": (dict(method="pcg", prec="fp64", persistent=True), 1e-9),
    "ff-persistent": (dict(method="pcg", prec="ff", persistent=True), 1e-9),
    "ff_bf16-persistent": (dict(method="pcg", prec="ff_bf16", persistent=True), 1e-8),
    "fp64-three-kernel-graph": (dict(method="pcg", prec="fp64", use_graph=True), 1e-9),
    "ff-three-kernel": (dict(method="pcg", prec="ff"), 1e-9),
    "fp64-chebyshev": (dict(method="pcg", prec="fp64", precond="chebyshev", poly_degree=4, use_graph=True), 1e-9),
    "ff-chebyshev": (dict(method="pcg", prec="ff", precond="chebyshev", poly_degree=4, use_graph=True), 1e-9),
    "ff-chebyshev-fp32-steps": (dict(method="pcg", prec="ff", precond="chebyshev", poly_degree=4, use_graph=True,
                                     poly_prec="fp32"), 1e-9),
    "ff-chebyshev-bf16-steps": (dict(method="pcg", prec="ff", precond="chebyshev", poly_degree=4, use_graph=True,
                                     poly_prec="bf16"), 1e-9),
    # the bench's headline solver with the bench's degree and ratio per dimension
    "ff-chebyshev-bf16-steps-bench-degree": (dict(method="pcg", prec="ff", precond="chebyshev", use_graph=True,
                                                  poly_prec="bf16"), 1e-9),
}
BENCH_DEGREE = {d: dict(poly_degree=bench.CHEB_DEGREE_FP32_STEPS[d], poly_ratio=bench.CHEB_RATIO_FP32_STEPS[d])
                for d in (2, 3)}
CASES_2D = list(SOLVERS)
CASES_3D = ["fp64-persistent", "ff-persistent", "ff-three-kernel", "fp64-chebyshev", "ff-chebyshev",
            "ff-chebyshev-fp32-steps", "ff-chebyshev-bf16-steps", "ff-chebyshev-bf16-steps-bench-degree"]


@pytest.mark.parametrize("solver", CASES_2D)
def test_2d_384_matches_oracle(truths, solver):
    mesh, hyb = gpu_problem("2d")
    assert mesh.nf > 8 * 152 * 256 and (mesh.nf + 255) // 256 > 3 * 152
    opts, tol = SOLVERS[solver]
    opts = dict(opts, **({"poly_ratio": 1000.0} if "chebyshev" in solver else {}))
    if "bench-degree" in solver:
        opts.update(BENCH_DEGREE[2])
    st, U, P = solve_recover(hyb, tol=1e-11, max_iter=400000, **opts)
    assert st["status"] == 0 and st["relres"] <= 1e-11
    Uo, Po = truths["2d"].result()[0]
    assert rel(U, Uo) <= tol and rel(P, Po) <= tol, (rel(U, Uo), rel(P, Po))


@pytest.mark.parametrize("inner", ["ff-jacobi", "ff-chebyshev-bf16-steps-bench-degree"])
def test_newton_384_matches_oracle(truths, inner):
    """The transient Newton step (flexible GMRES), its inner solves by the persistent
    Jacobi PCG or by the bench's float-float Chebyshev PCG with BF16 steps."""
    coords, elems, fbar, w = truth.newton_2d_inputs(NNEWTON)
    mesh = crhyb.cr_mesh_load(coords, elems)
    assert mesh.nf > 8 * 152 * 256
    fb = torch.from_numpy(fbar).cuda()
    hyb = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, 0.01, 1000.0, fb, conv="newton",
                                                       w=torch.from_numpy(w).cuda()), keep_fp32=False)
    pre = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, 0.01, 1000.0, fb), keep_fp32=False, keep_ff=True,
                             keep_bf16=True)
    extra = {} if inner == "ff-jacobi" else dict(precond="chebyshev", poly_prec="bf16", **BENCH_DEGREE[2])
    st, U, P = solve_recover(hyb, solver=lambda W: crhyb.cr_solve_preconditioned(hyb, pre, W, tol=1e-11,
                                                                                 prec="ff", max_iter=2000, **extra))
    assert st["status"] == 0 and st["relres"] <= 1e-11
    Uo, Po = truths["newton"].result()
    assert rel(U, Uo) <= 1e-9 and rel(P, Po) <= 1e-9, (rel(U, Uo), rel(P, Po))


def test_full_batch_largest_and_smallest_problems_match_oracle(truths):
    """The batched workload as the bench runs it (float-float, autotuned), every pair to
    1e-11; the largest problem (n = 234) and the smallest (n = 9) against the oracle."""
    probs = synth.batch_problems(count=64, nrhs=4, lo=8, hi=256, seed=2)
    hybs = []
    for q in probs:
        mesh = crhyb.cr_mesh_load(q["coords"], q["elems"])
        fb = torch.from_numpy(q["fbar"]).cuda()
        hybs.append(crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, q["nu"], q["mu"], fb), keep_fp32=False,
                                       keep_ff=True))
    batch = crhyb.cr_batch_create(hybs, prec="ff", autotune=True)
    Ws = [torch.zeros(4 * h.n, dtype=torch.float64, device="cuda") for h in hybs]
    stats = crhyb.cr_solve_batched(batch, Ws, tol=1e-11, max_iter=400000)
    assert all(s["status"] == 0 and s["relres"] <= 1e-11 for s in stats)
    sizes = [q["n"] for q in probs]
    for key, k in (("batch", _largest_batch_problem()), ("batch_small", int(np.argmin(sizes)))):
        h = hybs[k]
        ref = truths[key].result()
        for r in range(4):
            Wr = Ws[k][r * h.n:(r + 1) * h.n].contiguous()
            U = torch.zeros(h.n, dtype=torch.float64, device="cuda")
            P = torch.zeros(h.mesh.ne, dtype=torch.float64, device="cuda")
            crhyb.cr_recover_up(h, Wr, U, P, rhs=r, normalise_p=True)
            Uo, Po = ref[r]
            assert rel(U.cpu().numpy(), Uo) <= 1e-9 and rel(P.cpu().numpy(), Po) <= 1e-9, (key, r)


@pytest.mark.parametrize("solver", CASES_3D)
def test_3d_32cubed_matches_oracle(truths, solver):
    mesh, hyb = gpu_problem("3d")
    assert mesh.nf > 8 * 152 * 256 and (mesh.nf + 255) // 256 > 3 * 152
    opts, tol = SOLVERS[solver]
    opts = dict(opts, **({"poly_ratio": 100.0} if "chebyshev" in solver else {}))
    if "bench-degree" in solver:
        opts.update(BENCH_DEGREE[3])
    st, U, P = solve_recover(hyb, tol=1e-11, max_iter=400000, **opts)
    assert st["status"] == 0 and st["relres"] <= 1e-11
    Uo, Po, _ = truths["3d"].result()
    assert rel(U, Uo) <= tol and rel(P, Po) <= tol, (rel(U, Uo), rel(P, Po))


FORMS = ["rows1", "rows2", "staged"]


@pytest.mark.parametrize("form", FORMS)
def test_chebyshev_step_forms_match_oracle(truths, tmp_path, form):
    out = str(tmp_path / f"{form}.npz")
    here = os.path.dirname(os.path.abspath(__file__))
    path = os.pathsep.join([os.path.dirname(here), here] + [q for q in [os.environ.get("PYTHONPATH")] if q])
    env = dict(os.environ, CRHYB_CHEB_KERNEL=form, PYTHONPATH=path)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), form, out], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    got = np.load(out)
    for name, key in (("2d", "2d"), ("3d", "3d")):
        ref = truths[key].result()
        Uo, Po = (ref[0] if name == "2d" else ref[:2])
        for pp in ("fp32", "bf16"):
            U, P = got[f"{name}_{pp}_U"], got[f"{name}_{pp}_P"]
            assert got[f"{name}_{pp}_status"] == 0 and got[f"{name}_{pp}_relres"] <= 1e-11, (name, pp)
            assert rel(U, Uo) <= 1e-9 and rel(P, Po) <= 1e-9, (form, name, pp, rel(U, Uo), rel(P, Po))


def _child(form, out):
    """Solve the 2D and 3D cases with FP32 and BF16 Chebyshev steps in this process's form."""
    assert os.environ.get("CRHYB_CHEB_KERNEL") == form
    res = {}
    for name in ("2d", "3d"):
        mesh, hyb = gpu_problem(name)
        assert (mesh.nf + 255) // 256 > 5 * 152
        for pp in ("fp32", "bf16"):
            opts = dict(SOLVERS[f"ff-chebyshev-{pp}-steps"][0], poly_ratio=1000.0 if name == "2d" else 100.0)
            st, U, P = solve_recover(hyb, tol=1e-11, max_iter=400000, **opts)
            res.update({f"{name}_{pp}_U": U, f"{name}_{pp}_P": P, f"{name}_{pp}_status": st["status"],
                        f"{name}_{pp}_relres": st["relres"]})
    np.savez(out, **res)


if __name__ == "__main__":
    _child(sys.argv[1], sys.argv[2])
