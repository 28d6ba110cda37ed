"""Pins for the oracle's MINRES on the coupled system (Eq. 10 without
hybridisation, the comparison the paper draws against the hybrid method).

* The iterates equal those of SciPy's MINRES with the same preconditioner
  after a fixed number of steps (both minimise the same norm over the same
  Krylov space; only rounding differs).
* The running estimate |eta| is the preconditioned residual norm
  ||b - K x||_{M^{-1}} of the iterate.
* Run to a tight tolerance it reaches the direct solution of Eq. 10.
* The pressure part of the preconditioner is the diagonal of D diag(A)^{-1}
  D^t, computed here densely.
"""

import inspect

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import coupled, krylov, pipeline


def case(dim, n, mu, nu=1.0):
    if dim == 2:
        coords, elems = synth.mesh2d_square(n, perturb=0.2, seed=3)
    else:
        coords, elems = synth.mesh3d_kuhn(n)
    modes = synth.fourier_modes(dim, 1)
    fbar = synth.element_means(lambda x: synth.fourier_force(x, modes), coords, elems, order=3)
    ref = pipeline.direct(coords, elems, nu, mu, fbar, dense=True)
    return ref


def system(ref):
    A, D, R = ref["A"], ref["D"], ref["R"]
    K = coupled.saddle_matrix(A, D)
    b = np.concatenate([R, np.zeros(D.shape[0])])
    return A, D, K, b


def scipy_minres(K, b, minv, k):
    M = spla.LinearOperator(K.shape, matvec=lambda v: minv * v)
    kw = {"rtol": 0.0} if "rtol" in inspect.signature(spla.minres).parameters else {"tol": 0.0}
    x, _ = spla.minres(K, b, M=M, maxiter=k, **kw)
    return x


@pytest.mark.parametrize("dim,n,mu", [(2, 10, 1000.0), (2, 10, 0.0), (3, 2, 100.0)])
def test_iterates_equal_scipy_minres(dim, n, mu):
    ref = case(dim, n, mu)
    A, D, K, b = system(ref)
    minv = coupled.saddle_preconditioner(A, D)
    for k in (3, 17):
        ours, steps, _ = krylov.minres(K, b, minv, rtol=0.0, maxit=k)
        assert steps == k
        theirs = scipy_minres(K, b, minv, k)
        assert np.linalg.norm(ours - theirs) <= 1e-10 * np.linalg.norm(theirs)


def test_eta_is_the_preconditioned_residual_norm():
    ref = case(2, 8, 300.0)
    A, D, K, b = system(ref)
    minv = coupled.saddle_preconditioner(A, D)
    g1 = np.sqrt(np.dot(b, minv * b))
    for k in (1, 4, 11, 30):
        x, _, hist = krylov.minres(K, b, minv, rtol=0.0, maxit=k)
        r = b - K @ x
        assert abs(np.sqrt(np.dot(r, minv * r)) / g1 - hist[-1]) <= 1e-9 * max(hist[-1], 1e-3)


@pytest.mark.parametrize("mu", [1000.0, 0.0])
def test_minres_reaches_the_direct_solution(mu):
    ref = case(2, 9, mu)
    U, P, it, hist = coupled.solve_minres(ref["A"], ref["D"], ref["R"], rtol=1e-13)
    assert it > 10 and hist[-1] <= 1e-13
    assert np.linalg.norm(U - ref["U"].ravel()) <= 1e-10 * np.linalg.norm(ref["U"])
    vol = ref["geom"]["vol"]
    Pr = coupled.normalise_pressure(ref["P"], vol)
    assert np.linalg.norm(coupled.normalise_pressure(P, vol) - Pr) <= 1e-9 * np.linalg.norm(Pr)


def test_pressure_preconditioner_is_the_schur_diagonal():
    ref = case(2, 4, 50.0)
    A, D = ref["A"].toarray(), ref["D"].toarray()
    S = D @ np.diag(1.0 / np.diag(A)) @ D.T
    minv = coupled.saddle_preconditioner(ref["A"], ref["D"])
    N = A.shape[0]
    assert np.allclose(minv[:N], 1.0 / np.diag(A), rtol=1e-14, atol=0)
    assert np.allclose(minv[N:], 1.0 / np.diag(S), rtol=1e-13, atol=0)
