"""Pins for the oracle's Krylov solvers and iterative refinement.

Each solver is checked against a library direct solve (scipy's sparse LU)
on matrices of the kinds the method produces: the SPD hybridised matrix of
transient Stokes and the nonsymmetric one of a Newton step.  PCG's iterates
are also checked against SciPy's CG with the same preconditioner, and a GMRES
cycle against the minimal-residual iterate it is defined as.
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import hybrid, krylov, pipeline


def hybridised(dim, n, nu, mu, conv="none"):
    if dim == 2:
        coords, elems = synth.mesh2d_square(n, 0.2, 1)
    else:
        coords, elems = synth.mesh3d_kuhn(n)
    modes = synth.fourier_modes(dim, 1)
    fbar = synth.element_means(lambda x: synth.fourier_force(x, modes), coords, elems, order=3)
    w = None
    if conv != "none":
        from oracle import topology
        t = topology.build_faces(elems)
        w = synth.stream_velocity(coords[t["face_vertices"]].mean(axis=1), seed=3)
    topo, geom, A_K, D_K, R_K = pipeline.setup(coords, elems, nu, mu, fbar, conv, w)
    h = hybrid.hybridise(topo, A_K, D_K, R_K, mu)
    return h["G"], h["S"]


def test_pcg_matches_direct():
    G, S = hybridised(2, 12, 1.0, 1000.0)
    ref = spla.spsolve(G.tocsc(), S)
    x, it, hist = krylov.pcg(G, S, krylov.jacobi(G), rtol=1e-13)
    assert hist[-1] <= 1e-13 and it > 0
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-10
    # the recursive residual tracks the true residual
    assert np.linalg.norm(S - G @ x) / np.linalg.norm(S) < 1e-12


@pytest.mark.parametrize("dim,n,mu", [(2, 10, 1000.0), (3, 2, 100.0)])
def test_pcg_iterates_equal_scipy_cg(dim, n, mu):
    """After k steps the oracle's PCG iterate is SciPy's CG iterate with the
    same Jacobi preconditioner (the same recurrences; only rounding differs),
    which fixes alpha, beta and the preconditioned inner products."""
    import inspect
    G, S = hybridised(dim, n, 1.0, mu)
    minv = krylov.jacobi(G)
    M = spla.LinearOperator(G.shape, matvec=lambda v: minv * v)
    kw = {"rtol": 0.0, "atol": 0.0} if "rtol" in inspect.signature(spla.cg).parameters else {"tol": 0.0, "atol": 0.0}
    for k in (3, 20):
        ours, it, _ = krylov.pcg(G, S, minv, rtol=0.0, maxit=k)
        theirs, _ = spla.cg(G, S, M=M, maxiter=k, **kw)
        assert it == k
        assert np.linalg.norm(ours - theirs) <= 1e-10 * np.linalg.norm(theirs)


@pytest.mark.parametrize("m", [3, 6, 9])
def test_gmres_cycle_is_the_minimal_residual_iterate(m):
    """One cycle of m right-preconditioned GMRES steps from x = 0 gives the
    x in M K_m(G M, S) of least ||S - G x||_2 (the definition, solved here by a
    dense least-squares problem on an orthonormalised Krylov basis), and its
    running estimate is that iterate's relative residual."""
    G, S = hybridised(2, 8, 0.01, 100.0, "newton")
    minv = krylov.jacobi(G)
    A = G.toarray()
    x, it, hist = krylov.gmres(G, S, minv, restart=m, rtol=0.0, maxit=m)
    assert it == m
    basis, v = [], minv * S
    for _ in range(m):
        v = v / np.linalg.norm(v)
        basis.append(v)
        v = minv * (A @ v)
    Q, _ = np.linalg.qr(np.column_stack(basis))
    y, *_ = np.linalg.lstsq(A @ Q, S, rcond=None)
    xmin = Q @ y
    assert np.linalg.norm(x - xmin) <= 1e-9 * np.linalg.norm(xmin)
    assert abs(hist[-1] - np.linalg.norm(S - A @ x) / np.linalg.norm(S)) <= 1e-10


def test_pcg_zero_rhs_and_warm_start():
    G, S = hybridised(2, 6, 1.0, 100.0)
    x, it, _ = krylov.pcg(G, np.zeros_like(S), krylov.jacobi(G))
    assert it == 0 and not np.any(x)
    ref = spla.spsolve(G.tocsc(), S)
    x, it, _ = krylov.pcg(G, S, krylov.jacobi(G), x0=ref, rtol=1e-10)
    assert it <= 1


@pytest.mark.parametrize("conv,mu,restart", [("newton", 100.0, 30), ("oseen", 100.0, 30),
                                             ("newton", 0.0, 400), ("none", 0.0, 400)])
def test_gmres_matches_direct(conv, mu, restart):
    """Restarted GMRES on transient Newton/Oseen steps; full GMRES (restart >= N)
    on the steady (mu = 0) systems, where Jacobi-preconditioned GMRES(30)
    stagnates because the spectrum lies on both sides of zero."""
    G, S = hybridised(2, 8, 0.01 if conv != "none" else 1.0, mu, conv)
    assert restart == 30 or restart >= G.shape[0]
    ref = spla.spsolve(G.tocsc(), S)
    x, it, hist = krylov.gmres(G, S, krylov.jacobi(G), restart=restart, rtol=1e-12, maxit=5000)
    assert np.linalg.norm(S - G @ x) / np.linalg.norm(S) <= 1e-11
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-8


@pytest.mark.parametrize("inner", ["pcg", "gmres"])
def test_refinement_reaches_fp64_accuracy(inner):
    G, S = hybridised(2, 10, 1.0, 1000.0)
    ref = spla.spsolve(G.tocsc(), S)
    x, outer, tot, hist = krylov.refine(G, S, inner=inner, rtol=1e-13, inner_rtol=1e-4)
    assert hist[-1] <= 1e-13 and outer >= 2
    # error <= cond(G) * residual; cond(G) is a few thousand here
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-9


def test_hybrid_pipeline_methods_agree():
    coords, elems = synth.mesh2d_square(10, 0.2, 0)
    modes = synth.fourier_modes(2, 1)
    fbar = synth.element_means(lambda x: synth.fourier_force(x, modes), coords, elems, order=3)
    a = pipeline.hybrid(coords, elems, 1.0, 1000.0, fbar, method="direct")
    for m in ("pcg", "gmres", "ir-pcg"):
        b = pipeline.hybrid(coords, elems, 1.0, 1000.0, fbar, method=m, rtol=1e-13)
        assert np.linalg.norm(a["U"] - b["U"]) / np.linalg.norm(a["U"]) < 1e-10
