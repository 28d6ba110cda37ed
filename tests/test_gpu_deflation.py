"""Deflated PCG (cr_solve with a deflation space) and Ritz vectors from the
Lanczos connection of CG (cr_deflation_lanczos), against the CPU FP64 oracle.

* With the same vectors (the oracle's lowest eigenvectors of the pencil
  (G, diag G), rounded to FP32 as the library stores them), the GPU's FP64
  deflated PCG (Jacobi and Chebyshev) takes the oracle's deflated_pcg
  iteration count (within one) to 1e-10, and to 1e-12 reaches the direct
  solve within 1e-9 with its residual orthogonal to the space; float-float
  Chebyshev PCG (steps in float-float, FP32 or on BF16 values) deflated
  reaches the direct solve within 1e-9.
* The Ritz values of m FP64 PCG steps equal the oracle's lanczos_ritz values
  (same CG coefficients up to rounding), and the vectors span the same
  directions.
* Ritz vectors of one right-hand side cut the iterations of another.
* The dot products span more rows than one pass of their grid (2D 300^2).
* A vector in the span of the others is dropped; foreign systems and
  unsupported solvers are refused with CR_ERR_ARG.
"""

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import hybrid, krylov, pipeline
from paper_2101_03777_gb300 import crhyb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RATIO = {"cfg2": 1000.0, "cfg3": 100.0}
_CASES = {}


def case(name, n, nrhs=1):
    key = (name, n, nrhs)
    if key not in _CASES:
        p = synth.config_problem(name, n=n, nrhs=nrhs)
        Gs, Ss = [], []
        for r in range(nrhs):
            topo, geom, A_K, D_K, R_K = pipeline.setup(p["coords"], p["elems"], p["nu"], p["mu"], p["fbar"][r],
                                                       p["conv"])
            h = hybrid.hybridise(topo, A_K, D_K, R_K, p["mu"])
            Gs.append(h["G"].tocsr())
            Ss.append(h["S"])
        mesh = crhyb.cr_mesh_load(p["coords"], p["elems"])
        fb = torch.from_numpy(p["fbar"]).cuda()
        hyb = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, p["nu"], p["mu"], fb), keep_fp32=True,
                                 keep_bf16=True, keep_ff=True)
        _CASES[key] = (Gs[0], Ss, mesh, hyb, p)
    return _CASES[key]


def low_modes(G, k):
    """The k lowest eigenvectors of G v = lambda diag(G) v, rounded to FP32."""
    _, vecs = spla.eigsh(G.tocsc(), k=k, M=sp.diags(G.diagonal()).tocsc(), sigma=0, which="LM")
    return np.ascontiguousarray(vecs.T.astype(np.float32).astype(np.float64))


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_solve(hyb, rhs=0, **opts):
    W = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    st = crhyb.cr_solve(hyb, W, rhs=rhs, **opts)
    return st, W.cpu().numpy()


@pytest.mark.parametrize("name,n", [("cfg2", 24), ("cfg3", 4)])
@pytest.mark.parametrize("precond", ["jacobi", "chebyshev"])
@pytest.mark.parametrize("graph", [False, True])
def test_fp64_deflated_pcg_matches_oracle(name, n, precond, graph):
    G, Ss, mesh, hyb, _ = case(name, n)
    S = Ss[0]
    V = low_modes(G, 4)
    d = crhyb.cr_deflation_create(hyb, V)
    assert d.k == 4 and np.array_equal(d.vectors(), V)
    minv = krylov.jacobi(G)
    if precond == "jacobi":
        pc = lambda r: minv * r   # noqa: E731
        extra = {}
    else:
        lmax = krylov.gershgorin_bound(G, minv)
        pc = lambda r: krylov.chebyshev_apply(G, minv, r, 4, lmax, RATIO[name])   # noqa: E731
        extra = dict(poly_degree=4, poly_ratio=RATIO[name])
    _, it, _ = krylov.deflated_pcg(G, S, pc, V.T, rtol=1e-10)
    st, W = gpu_solve(hyb, prec="fp64", precond=precond, tol=1e-10, deflation=d, use_graph=graph, check_every=7,
                      **extra)
    assert st["status"] == 0 and st["relres"] <= 1e-10
    assert abs(st["iterations"] - it) <= 1, (st["iterations"], it)
    # fewer iterations than without deflation
    st0, _ = gpu_solve(hyb, prec="fp64", precond=precond, tol=1e-10, **extra)
    assert st["iterations"] < st0["iterations"]
    # W: to 1e-12 against the direct solve, the residual orthogonal to the space
    st, W = gpu_solve(hyb, prec="fp64", precond=precond, tol=1e-12, deflation=d, use_graph=graph, **extra)
    assert st["status"] == 0 and rel(W, spla.spsolve(G.tocsc(), S)) <= 1e-9
    r = S - G @ W
    assert np.abs(V @ r).max() <= 1e-11 * np.abs(V).sum(axis=1).max() * np.linalg.norm(S)


@pytest.mark.parametrize("poly_prec", ["same", "fp32", "bf16"])
@pytest.mark.parametrize("name,n", [("cfg2", 24), ("cfg3", 4)])
def test_float_float_deflated_chebyshev_reaches_the_direct_solve(name, n, poly_prec):
    G, Ss, mesh, hyb, _ = case(name, n)
    S = Ss[0]
    ref = spla.spsolve(G.tocsc(), S)
    d = crhyb.cr_deflation_create(hyb, low_modes(G, 4))
    opts = dict(prec="ff", precond="chebyshev", poly_degree=4, poly_ratio=RATIO[name], poly_prec=poly_prec,
                tol=1e-12, use_graph=True)
    st, W = gpu_solve(hyb, deflation=d, **opts)
    assert st["status"] == 0 and st["relres"] <= 1e-12
    assert rel(W, ref) <= 1e-9
    st0, _ = gpu_solve(hyb, **opts)
    assert st["iterations"] < st0["iterations"]


@pytest.mark.parametrize("precond", ["jacobi", "chebyshev"])
def test_ritz_values_match_oracle(precond):
    G, Ss, mesh, hyb, _ = case("cfg2", 24)
    S = Ss[0]
    minv = krylov.jacobi(G)
    if precond == "jacobi":
        pc = lambda r: minv * r   # noqa: E731
        extra = {}
    else:
        lmax = krylov.gershgorin_bound(G, minv)
        pc = lambda r: krylov.chebyshev_apply(G, minv, r, 4, lmax, 1000.0)   # noqa: E731
        extra = dict(poly_degree=4, poly_ratio=1000.0)
    th_o, Y_o, _ = krylov.lanczos_ritz(G, S, pc, 40, 4)
    d, th = crhyb.cr_deflation_lanczos(hyb, 40, 4, precond=precond, **extra)
    assert d.k == 4
    assert np.allclose(th, th_o, rtol=1e-7, atol=0), (th, th_o)
    Y = d.vectors()
    for j in range(4):
        yo = Y_o[:, j] / np.linalg.norm(Y_o[:, j])
        yg = Y[j] / np.linalg.norm(Y[j])
        assert abs(yo @ yg) >= 1 - 1e-5, j


@pytest.mark.parametrize("m,poly_prec,gain", [(120, "same", 0.8), (120, "fp32", 0.8), (120, "bf16", 0.9),
                                               (300, "bf16", 0.7)])
def test_ritz_vectors_of_one_rhs_speed_up_another(m, poly_prec, gain):
    """2D 64^2, two right-hand sides: 8 Ritz vectors from m FP64 Chebyshev-PCG steps on
    the first cut the float-float Chebyshev PCG of the second, which still reaches the
    direct solve.  From 120 steps (a third of a solve) the space misses the isolated
    lowest mode, which the preconditioner amplifies in z: the dot products and the
    projection must then be exact for the FP32 z and V (they are FP64), or they feed
    components along V back into every direction and the gain is lost.  Measured:
    322-323 -> 246 / 247 / 277 iterations with float-float, FP32 and BF16 steps (FP64
    PCG: 320 -> 244; the BF16 steps' rounded G makes the space less invariant);
    from 300 steps, BF16: 323 -> 173."""
    G, Ss, mesh, hyb, _ = case("cfg2", 64, nrhs=2)
    cheb = dict(precond="chebyshev", poly_degree=4, poly_ratio=1000.0)
    d, th = crhyb.cr_deflation_lanczos(hyb, m, 8, rhs=0, **cheb)
    assert d.k >= 6 and np.all(np.diff(th) >= 0) and th[0] > 0
    opts = dict(prec="ff", poly_prec=poly_prec, tol=1e-12, use_graph=True, **cheb)
    st0, _ = gpu_solve(hyb, rhs=1, **opts)
    st, W = gpu_solve(hyb, rhs=1, deflation=d, **opts)
    assert st["status"] == 0 and st["relres"] <= 1e-12
    # W's error is about 700 times its relative residual on this mesh (measured: 7e-9 at 1e-11)
    assert rel(W, spla.spsolve(G.tocsc(), Ss[1])) <= 1e-8
    assert st["iterations"] < gain * st0["iterations"], (st["iterations"], st0["iterations"])


def test_dot_products_over_several_grid_passes():
    """2D 300^2: 538,800 unknowns, more than the 262,144 rows of one pass of the deflation
    kernels' grid.  FP64 Jacobi PCG deflated by 6 Ritz vectors reaches the undeflated
    solution, and the residual of the returned W is orthogonal to the space."""
    p = synth.config_problem("cfg2", n=300)
    mesh = crhyb.cr_mesh_load(p["coords"], p["elems"])
    hyb = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, p["nu"], p["mu"], torch.from_numpy(p["fbar"]).cuda()))
    assert hyb.n > 1024 * 256
    d, _ = crhyb.cr_deflation_lanczos(hyb, 60, 6)
    st0, W0 = gpu_solve(hyb, prec="fp64", tol=1e-11, use_graph=True)
    st, W = gpu_solve(hyb, prec="fp64", tol=1e-11, use_graph=True, deflation=d)
    assert st["status"] == 0 and st["relres"] <= 1e-11 and st["iterations"] < st0["iterations"]

    def velocity(Wn):   # the recovered U is far better conditioned than W
        U = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
        P = torch.zeros(mesh.ne, dtype=torch.float64, device="cuda")
        crhyb.cr_recover_up(hyb, torch.from_numpy(Wn).cuda(), U, P, normalise_p=True)
        return U.cpu().numpy()
    assert rel(velocity(W), velocity(W0)) <= 1e-9
    Gx = torch.empty(hyb.n, dtype=torch.float64, device="cuda")
    crhyb.cr_apply_G(hyb, torch.from_numpy(W).cuda(), Gx)
    _, _, S = crhyb.cr_hybrid_export(hyb)
    r = S[0].ravel() - Gx.cpu().numpy()
    V = d.vectors()
    assert np.abs(V @ r).max() <= 1e-8 * np.abs(V).sum(axis=1).max() * np.linalg.norm(S[0])


def test_dependent_vectors_are_dropped():
    G, Ss, mesh, hyb, _ = case("cfg2", 24)
    V = low_modes(G, 3)
    V4 = np.ascontiguousarray(np.vstack([V[:2], V[0] + V[1], V[2:]]))   # the third is the sum of the first two
    d = crhyb.cr_deflation_create(hyb, V4)
    assert d.k == 3 and np.array_equal(d.vectors(), V)


def test_foreign_systems_and_unsupported_solvers_are_refused():
    G, Ss, mesh, hyb, p = case("cfg2", 24)
    d = crhyb.cr_deflation_create(hyb, low_modes(G, 2))
    fb = torch.from_numpy(p["fbar"]).cuda()
    other = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, p["nu"], 0.5 * p["mu"], fb), keep_ff=True)
    W = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    for h, opts in ((other, dict(prec="fp64")),                     # another G
                    (hyb, dict(prec="ff")),                         # float-float Jacobi
                    (hyb, dict(prec="ff_bf16", precond="chebyshev")),
                    (hyb, dict(prec="fp64", method="gmres"))):
        with pytest.raises(crhyb.CrError) as ei:
            crhyb.cr_solve(h, W, deflation=d, **opts)
        assert ei.value.name == "CR_ERR_ARG"
    # the same G in a new hybridised system (a later time step) is accepted
    same = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, p["nu"], p["mu"], fb))
    assert crhyb.cr_solve(same, W, prec="fp64", tol=1e-10, deflation=d)["status"] == 0
    for m, k in ((3, 4), (40, 0), (40, 17)):
        with pytest.raises(crhyb.CrError) as ei:
            crhyb.cr_deflation_lanczos(hyb, m, k)
        assert ei.value.name == "CR_ERR_ARG"
    with pytest.raises(crhyb.CrError):
        crhyb.cr_deflation_create(hyb, np.zeros((2, hyb.n)))   # V^t G V = 0


def test_recorded_solve_gives_the_oracle_ritz_values():
    """cr_solve_ritz, FP64 Jacobi PCG: the solve is cr_solve's (same W, same iterations) and
    the Ritz values of its first 40 iterations' record equal the oracle's lanczos_ritz over
    the same 39 steps (T closes one step fewer than the vectors recorded)."""
    G, Ss, mesh, hyb, _ = case("cfg2", 24)
    S = Ss[0]
    minv = krylov.jacobi(G)
    W = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    st, d, th = crhyb.cr_solve_ritz(hyb, W, 40, 4, prec="fp64", tol=1e-10, use_graph=True)
    st0, W0 = gpu_solve(hyb, prec="fp64", tol=1e-10, use_graph=True)
    assert st["status"] == 0 and st["iterations"] == st0["iterations"] and np.array_equal(W.cpu().numpy(), W0)
    th_o, Y_o, _ = krylov.lanczos_ritz(G, S, lambda r: minv * r, 39, 4)
    assert d.k == 4 and np.allclose(th, th_o, rtol=1e-7, atol=0), (th, th_o)
    Y = d.vectors()
    for j in range(4):
        assert abs((Y_o[:, j] / np.linalg.norm(Y_o[:, j])) @ (Y[j] / np.linalg.norm(Y[j]))) >= 1 - 1e-5, j


def test_recorded_float_float_solve_deflates_the_next_right_hand_side():
    """The time-loop pattern: the float-float Chebyshev PCG (BF16 steps) of the first
    right-hand side records 150 iterations; its 8 Ritz vectors cut the iterations of the
    second right-hand side, which still reaches the direct solve."""
    G, Ss, mesh, hyb, _ = case("cfg2", 64, nrhs=2)
    opts = dict(prec="ff", precond="chebyshev", poly_degree=8, poly_ratio=1000.0, poly_prec="bf16", tol=1e-12,
                use_graph=True)
    W = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    st, d, th = crhyb.cr_solve_ritz(hyb, W, 150, 8, rhs=0, **opts)
    assert st["status"] == 0 and st["relres"] <= 1e-12 and d.k >= 6 and th[0] > 0
    assert rel(W.cpu().numpy(), spla.spsolve(G.tocsc(), Ss[0])) <= 1e-8
    st0, _ = gpu_solve(hyb, rhs=1, **opts)
    st1, W1 = gpu_solve(hyb, rhs=1, deflation=d, **opts)
    assert st1["status"] == 0 and st1["relres"] <= 1e-12
    assert rel(W1, spla.spsolve(G.tocsc(), Ss[1])) <= 1e-8
    assert st1["iterations"] < 0.85 * st0["iterations"], (st1["iterations"], st0["iterations"])


def test_recorded_solve_arguments():
    G, Ss, mesh, hyb, _ = case("cfg2", 24)
    W = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    d = crhyb.cr_deflation_create(hyb, low_modes(G, 2))
    for m, k, opts in ((3, 4, dict(prec="fp64")), (40, 0, dict(prec="fp64")), (40, 4, dict(prec="ff")),
                       (40, 4, dict(prec="fp64", method="gmres")), (40, 4, dict(prec="fp64", deflation=d))):
        with pytest.raises(crhyb.CrError) as ei:
            crhyb.cr_solve_ritz(hyb, W, m, k, **opts)
        assert ei.value.name == "CR_ERR_ARG"
