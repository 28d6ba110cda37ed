"""Pins for the oracle's deflated CG (krylov.deflated_pcg), the next lever
after the Chebyshev preconditioner for G's isolated low eigenvalues.

* With no deflation vectors it is the oracle's PCG, iterate for iterate.
* Every residual stays orthogonal to the deflation vectors.
* On a diagonal system, deflating coordinate directions splits the problem:
  the deflated components are exact from the start and the rest follows
  plain CG on the remaining diagonal, step for step (the definition).
* It reaches the direct solution of G W = S, and deflating the lowest modes
  of M^{-1} G (with the Chebyshev or the Jacobi preconditioner) takes fewer
  iterations.
"""

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import hybrid, krylov, pipeline


def hybrid_system(n):
    p = synth.config_problem("cfg2", n=n)
    topo, geom, A_K, D_K, R_K = pipeline.setup(p["coords"], p["elems"], p["nu"], p["mu"], p["fbar"][0], p["conv"])
    h = hybrid.hybridise(topo, A_K, D_K, R_K, p["mu"])
    return h["G"].tocsr(), h["S"]


def test_no_vectors_is_pcg():
    G, S = hybrid_system(10)
    minv = krylov.jacobi(G)
    for k in (5, 40):
        x1, it1, h1 = krylov.pcg(G, S, minv, rtol=0.0, maxit=k)
        x2, it2, h2 = krylov.deflated_pcg(G, S, lambda r: minv * r, np.zeros((G.shape[0], 0)), rtol=0.0, maxit=k)
        assert it1 == it2 == k
        assert np.linalg.norm(x1 - x2) <= 1e-12 * np.linalg.norm(x1)


def test_residuals_stay_orthogonal_to_the_vectors():
    G, S = hybrid_system(10)
    minv = krylov.jacobi(G)
    V = np.random.default_rng(5).standard_normal((G.shape[0], 3))
    for k in (1, 7, 30):
        x, _, _ = krylov.deflated_pcg(G, S, lambda r: minv * r, V, rtol=0.0, maxit=k)
        r = S - G @ x
        assert np.abs(V.T @ r).max() <= 1e-9 * np.linalg.norm(V, axis=0).max() * np.linalg.norm(S)


def test_diagonal_system_splits():
    rng = np.random.default_rng(9)
    lam = np.sort(rng.uniform(1e-3, 1.0, 40))
    G = sp.diags(lam).tocsr()
    b = rng.standard_normal(40)
    k = 5
    V = np.eye(40)[:, :k]                     # the five smallest eigenvalues deflated
    for steps in (3, 12):
        x, it, _ = krylov.deflated_pcg(G, b, lambda r: r, V, rtol=0.0, maxit=steps)
        assert np.allclose(x[:k], b[:k] / lam[:k], rtol=1e-12, atol=0)
        y, _, _ = krylov.pcg(sp.diags(lam[k:]).tocsr(), b[k:], np.ones(40 - k), rtol=0.0, maxit=steps)
        assert np.linalg.norm(x[k:] - y) <= 1e-10 * np.linalg.norm(y)


@pytest.mark.parametrize("cheb", [False, True])
def test_low_modes_deflated_reach_the_solution_sooner(cheb):
    G, S = hybrid_system(24)
    minv = krylov.jacobi(G)
    ref = spla.spsolve(G.tocsc(), S)
    if cheb:
        lmax = krylov.gershgorin_bound(G, minv)
        precond = lambda r: krylov.chebyshev_apply(G, minv, r, 4, lmax, 1000.0)
    else:
        precond = lambda r: minv * r
    _, vecs = spla.eigsh(G.tocsc(), k=4, M=sp.diags(G.diagonal()).tocsc(), sigma=0, which="LM")
    x0, it0, _ = krylov.deflated_pcg(G, S, precond, np.zeros((G.shape[0], 0)), rtol=1e-12)
    x, it, hist = krylov.deflated_pcg(G, S, precond, vecs, rtol=1e-12)
    assert hist[-1] <= 1e-12
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    assert it < it0


# ---- Ritz vectors from the Lanczos connection of CG (krylov.lanczos_ritz) ----

def test_lanczos_matrix_is_q_transpose_g_q():
    """T from the CG coefficients equals Q^t G Q formed from the stored vectors, and
    Q^t M Q = I for the Jacobi preconditioner (M = diag(G)): catches a wrong sign of
    the off-diagonal, a dropped beta/alpha term and unnormalised vectors."""
    G, S = hybrid_system(10)
    minv = krylov.jacobi(G)
    m = 12
    # the Lanczos vectors again, as the oracle stores them, to form Q^t G Q directly
    r = S.copy()
    z = minv * r
    p = z.copy()
    rz = r @ z
    Q = []
    for _ in range(m):
        Q.append(z / np.sqrt(rz))
        q = G @ p
        a = rz / (p @ q)
        r = r - a * q
        z = minv * r
        rzn = r @ z
        p = z + (rzn / rz) * p
        rz = rzn
    Q = np.array(Q).T
    theta, Y, T = krylov.lanczos_ritz(G, S, lambda v: minv * v, m, 4)
    QGQ = Q.T @ (G @ Q)
    assert T.shape == (m, m)
    assert np.abs(QGQ - T).max() <= 1e-8 * np.abs(T).max()
    assert np.abs(Q.T @ (G.diagonal()[:, None] * Q) - np.eye(m)).max() <= 1e-8
    # Galerkin condition of the returned Ritz pairs
    for j in range(len(theta)):
        res = G @ Y[:, j] - theta[j] * G.diagonal() * Y[:, j]
        assert np.abs(Q.T @ res).max() <= 1e-8 * np.linalg.norm(G.diagonal() * Y[:, j]) * max(theta[j], 1.0)


def test_full_lanczos_gives_the_exact_smallest_eigenvalues():
    """On a diagonal system with n distinct eigenvalues, n CG steps from a vector with
    every component give T with exactly those eigenvalues; the k smallest come back
    first, and the Ritz vectors are the coordinate vectors (up to sign)."""
    rng = np.random.default_rng(4)
    lam = np.sort(rng.uniform(0.5, 20.0, 12))
    G = sp.diags(lam).tocsr()
    b = rng.uniform(0.5, 1.5, 12)
    theta, Y, T = krylov.lanczos_ritz(G, b, lambda r: r, 12, 3)
    assert np.allclose(theta, lam[:3], rtol=1e-9, atol=0)
    assert np.allclose(np.abs(Y[:3, :3]), np.eye(3), atol=1e-6)
    assert np.allclose(np.linalg.eigvalsh(T), lam, rtol=1e-9, atol=0)


def test_jacobi_preconditioned_ritz_values_are_generalised_eigenvalues():
    """With M = diag(G) and enough steps, the smallest Ritz values reach the smallest
    eigenvalues of the pencil (G, M) (dense solve on a small hybridised system)."""
    import scipy.linalg as sla
    G, S = hybrid_system(6)
    minv = krylov.jacobi(G)
    Gd = G.toarray()
    ev = sla.eigh(Gd, np.diag(G.diagonal()), eigvals_only=True)
    theta, Y, _ = krylov.lanczos_ritz(G, S, lambda v: minv * v, 80, 2)
    assert np.allclose(theta, ev[:2], rtol=1e-6, atol=0)


def test_ritz_vectors_of_one_solve_deflate_the_next():
    """The Ritz vectors of a short Chebyshev-PCG run on one right-hand side, deflated in
    the solve of another right-hand side with the same G, reach its solution in fewer
    iterations."""
    G, S = hybrid_system(24)
    minv = krylov.jacobi(G)
    lmax = krylov.gershgorin_bound(G, minv)
    precond = lambda r: krylov.chebyshev_apply(G, minv, r, 4, lmax, 1000.0)   # noqa: E731
    _, Y, _ = krylov.lanczos_ritz(G, S, precond, 60, 8)
    b2 = np.random.default_rng(3).standard_normal(G.shape[0])
    ref = spla.spsolve(G.tocsc(), b2)
    _, it0, _ = krylov.deflated_pcg(G, b2, precond, np.zeros((G.shape[0], 0)), rtol=1e-10)
    x, it, _ = krylov.deflated_pcg(G, b2, precond, Y, rtol=1e-10)
    assert np.linalg.norm(x - ref) <= 1e-7 * np.linalg.norm(ref)
    assert it < 0.85 * it0, (it, it0)
