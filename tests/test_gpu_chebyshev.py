"""The Chebyshev-preconditioned PCG of cr_solve (precond = CHEBYSHEV; FP64, and
float-float with FP64 reliable updates) against the CPU FP64 oracle.

* W reaches the oracle's direct solve of G W = S (1e-9 relative L2 after a
  solve to a relative residual of 1e-12), in 2D and 3D, for several degrees
  and interval ratios.
* The CG iteration count equals the oracle's Chebyshev PCG count for the same
  degree and ratio (same algorithm, same Gershgorin bound; rounding moves it
  by at most a few).
* Graph replay, plain launches and the persistent flag (ignored by this
  preconditioner) give bit-identical W: every reduction is deterministic.
* Bad options are refused with CR_ERR_ARG.
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import hybrid, krylov, pipeline
from paper_2101_03777_gb300 import crhyb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


_CASES = {}


def case(name, n):
    if (name, n) not in _CASES:
        p = synth.config_problem(name, n=n)
        topo, geom, A_K, D_K, R_K = pipeline.setup(p["coords"], p["elems"], p["nu"], p["mu"], p["fbar"][0],
                                                   p["conv"])
        h = hybrid.hybridise(topo, A_K, D_K, R_K, p["mu"])
        G, S = h["G"].tocsr(), h["S"]
        mesh = crhyb.cr_mesh_load(p["coords"], p["elems"])
        fb = torch.from_numpy(p["fbar"]).cuda()
        hyb = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, p["nu"], p["mu"], fb), keep_fp32=True,
                                 keep_bf16=True, keep_ff=True, keep_ff_bf16=True)
        _CASES[(name, n)] = (G, S, spla.spsolve(G.tocsc(), S), mesh, hyb)
    return _CASES[(name, n)]


def solve(hyb, **opts):
    W = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    opts.setdefault("prec", "fp64")
    st = crhyb.cr_solve(hyb, W, method="pcg", precond="chebyshev", **opts)
    return st, W.cpu().numpy()


@pytest.mark.parametrize("name,n,degree,ratio", [("cfg2", 29, 4, 100.0), ("cfg2", 29, 2, 1000.0),
                                                 ("cfg2", 29, 8, 1000.0), ("cfg3", 4, 4, 100.0),
                                                 ("cfg3", 4, 3, 30.0)])
def test_matches_the_oracle(name, n, degree, ratio):
    G, S, ref, mesh, hyb = case(name, n)
    st, W = solve(hyb, tol=1e-12, poly_degree=degree, poly_ratio=ratio, use_graph=True)
    assert st["status"] == 0 and st["relres"] <= 1e-11   # the true residual; CG stops on the recursive one
    assert rel(W, ref) <= 1e-9
    _, it, _ = krylov.chebyshev_pcg(G, S, krylov.jacobi(G), degree, ratio, rtol=1e-12)
    assert abs(st["iterations"] - it) <= max(3, 0.02 * it)
    # fewer CG iterations than Jacobi-PCG
    Wj = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    stj = crhyb.cr_solve(hyb, Wj, method="pcg", prec="fp64", tol=1e-12)
    assert st["iterations"] < stj["iterations"]


@pytest.mark.parametrize("prec,tol", [("ff", 1e-9), ("ff_bf16", 1e-8)])
@pytest.mark.parametrize("name,n,degree,ratio", [("cfg2", 29, 4, 1000.0), ("cfg2", 29, 8, 300.0),
                                                 ("cfg3", 4, 4, 100.0)])
def test_float_float_matches_the_oracle(prec, tol, name, n, degree, ratio):
    """The same Chebyshev PCG in float-float with FP64 reliable updates: W within the
    parity tolerance of the direct solve, and about the oracle's CG iteration count
    (the reliable updates continue the search direction)."""
    G, S, ref, mesh, hyb = case(name, n)
    st, W = solve(hyb, prec=prec, tol=1e-12, poly_degree=degree, poly_ratio=ratio, use_graph=True)
    assert st["status"] == 0 and st["relres"] <= 1e-12 and st["outer"] >= 1
    assert rel(W, ref) <= tol
    _, it, _ = krylov.chebyshev_pcg(G, S, krylov.jacobi(G), degree, ratio, rtol=1e-12)
    assert st["iterations"] <= 1.3 * it + 5, (st["iterations"], it)


@pytest.mark.parametrize("poly_prec", ["fp32", "bf16"])
@pytest.mark.parametrize("name,n,ratio", [("cfg2", 29, 1000.0), ("cfg3", 4, 100.0)])
def test_reduced_precision_preconditioner_steps(poly_prec, name, n, ratio):
    """The Chebyshev steps in FP32 on FP32 or BF16 values of G (the preconditioner
    only): W still reaches the direct solve at the float-float tolerance, and the CG
    iteration count stays near the oracle's FP64 count (the polynomial of the rounded
    G is still a symmetric positive definite preconditioner)."""
    G, S, ref, mesh, hyb = case(name, n)
    st, W = solve(hyb, prec="ff", tol=1e-12, poly_degree=4, poly_ratio=ratio, poly_prec=poly_prec, use_graph=True)
    assert st["status"] == 0 and st["relres"] <= 1e-12
    assert rel(W, ref) <= 1e-9
    _, it, _ = krylov.chebyshev_pcg(G, S, krylov.jacobi(G), 4, ratio, rtol=1e-12)
    assert st["iterations"] <= 1.5 * it + 5, (st["iterations"], it)


def test_float_float_graph_and_plain_agree():
    G, S, ref, mesh, hyb = case("cfg2", 29)
    st_g, W_g = solve(hyb, prec="ff", tol=1e-11, use_graph=True, check_every=5)
    st_p, W_p = solve(hyb, prec="ff", tol=1e-11, use_graph=False, profile=True)
    assert st_g["iterations"] == st_p["iterations"] and np.array_equal(W_g, W_p)
    assert st_p["spmv_launches"] >= st_p["iterations"] - st_p["outer"] - 1 and st_p["spmv_ms"] > 0.0


def test_graph_plain_and_persistent_flag_agree():
    G, S, ref, mesh, hyb = case("cfg2", 29)
    st_g, W_g = solve(hyb, tol=1e-11, use_graph=True, check_every=7)
    st_p, W_p = solve(hyb, tol=1e-11, use_graph=False, profile=True)
    st_q, W_q = solve(hyb, tol=1e-11, persistent=True)
    assert st_g["iterations"] == st_p["iterations"] == st_q["iterations"]
    assert np.array_equal(W_g, W_p) and np.array_equal(W_g, W_q)
    # profile: the Chebyshev steps of every counted iteration were timed
    assert st_p["spmv_launches"] >= st_p["iterations"] - 1 and st_p["spmv_ms"] > 0.0


def test_default_degree_and_ratio():
    G, S, ref, mesh, hyb = case("cfg2", 29)
    st0, W0 = solve(hyb, tol=1e-11)
    st1, W1 = solve(hyb, tol=1e-11, poly_degree=4, poly_ratio=100.0)
    assert st0["iterations"] == st1["iterations"] and np.array_equal(W0, W1)


def test_zero_source_and_iteration_limit():
    G, S, ref, mesh, hyb = case("cfg2", 29)
    st, W = solve(hyb, tol=1e-12, max_iter=5, raise_on_error=False)
    assert st["status_name"] == "CR_ERR_NOT_CONVERGED" and st["iterations"] == 5
    p = synth.config_problem("cfg2", n=6)
    m0 = crhyb.cr_mesh_load(p["coords"], p["elems"])
    fb = torch.zeros(1, m0.ne, 2, dtype=torch.float64, device="cuda")
    h0 = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(m0, 1.0, 100.0, fb), keep_fp32=False)
    st, W = solve(h0, tol=1e-10)
    assert st["status"] == 0 and not W.any()


def test_bad_options_are_refused():
    G, S, ref, mesh, hyb = case("cfg2", 29)
    W = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    bad = [dict(prec="mixed"), dict(method="gmres"), dict(poly_degree=1), dict(poly_degree=33),
           dict(poly_prec="fp32"),   # reduced-precision steps apply to the float-float PCG only
           dict(poly_ratio=0.5), dict(poly_ratio=1.0)]
    for b in bad:
        o = {"method": "pcg", "prec": "fp64", "precond": "chebyshev", "tol": 1e-10, **b}
        with pytest.raises(crhyb.CrError) as ei:
            crhyb.cr_solve(hyb, W, **o)
        assert ei.value.name == "CR_ERR_ARG", b
    with pytest.raises(crhyb.CrError) as ei:   # FP32 steps under an FP64 inner solve
        crhyb.cr_solve_preconditioned(hyb, hyb, W, tol=1e-10, prec="fp64", precond="chebyshev", poly_prec="fp32")
    assert ei.value.name == "CR_ERR_ARG"
