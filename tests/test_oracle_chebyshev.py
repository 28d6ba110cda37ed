"""Pins for the oracle's Chebyshev polynomial preconditioner and the CG that
uses it (a stronger preconditioner for G than Jacobi; the paper's
preconditioning axis, Section 4).

* On an eigenvector v of M^{-1} G (eigenvalue lam) the preconditioner is the
  scalar (1 - T_k((theta - lam)/delta) / T_k(theta/delta)) / lam, the closed
  form of k Chebyshev steps from zero, evaluated here with NumPy's Chebyshev
  series: this fixes every coefficient of the three-term recurrence.
* The Gershgorin bound is above the spectrum of M^{-1} G, and with it the
  preconditioner is symmetric positive definite (with a bound below the
  spectrum it is not, which the test also shows).
* Degree 1 is Jacobi scaled by 1/theta, so CG takes the Jacobi-PCG iterates.
* The preconditioned CG reaches the direct solution of G W = S.
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spla
from numpy.polynomial import chebyshev as npcheb

import synth
from oracle import hybrid, krylov, pipeline


def hybrid_system(name, n):
    p = synth.config_problem(name, n=n)
    topo, geom, A_K, D_K, R_K = pipeline.setup(p["coords"], p["elems"], p["nu"], p["mu"], p["fbar"][0], p["conv"])
    h = hybrid.hybridise(topo, A_K, D_K, R_K, p["mu"])
    return h["G"].tocsr(), h["S"]


def closed_form(lam, degree, lmax, ratio):
    a, b = lmax / ratio, lmax
    theta, delta = 0.5 * (b + a), 0.5 * (b - a)
    tk = [0.0] * degree + [1.0]
    return (1.0 - npcheb.chebval((theta - lam) / delta, tk) / npcheb.chebval(theta / delta, tk)) / lam


@pytest.mark.parametrize("degree", [1, 2, 3, 5, 8])
def test_eigenvectors_get_the_closed_form(degree):
    rng = np.random.default_rng(11)
    n = 14
    X = rng.standard_normal((n, n))
    G = X @ X.T + 0.3 * np.eye(n)
    minv = rng.uniform(0.5, 2.0, n)
    s = np.sqrt(minv)
    lam, Q = np.linalg.eigh(s[:, None] * G * s[None, :])   # spectrum of M^{-1} G
    lmax, ratio = 1.01 * lam[-1], 25.0                        # some eigenvalues fall below lmax/ratio
    assert lam[0] < lmax / ratio
    for i in range(n):
        v = s * Q[:, i]                 # M^{-1} G v = lam v
        r = v / minv                    # M^{-1} r = v
        z = krylov.chebyshev_apply(G, minv, r, degree, lmax, ratio)
        want = closed_form(lam[i], degree, lmax, ratio) * v
        assert np.linalg.norm(z - want) <= 1e-10 * np.linalg.norm(want)


@pytest.mark.parametrize("name,n", [("cfg2", 5), ("cfg3", 2)])
def test_bound_and_spd(name, n):
    G, _ = hybrid_system(name, n)
    minv = krylov.jacobi(G)
    Gd = G.toarray()
    s = np.sqrt(minv)
    lam = np.linalg.eigvalsh(s[:, None] * Gd * s[None, :])
    bound = krylov.gershgorin_bound(G, minv)
    assert lam[-1] <= bound
    N = G.shape[0]
    for degree in (2, 4, 7):
        P = np.column_stack([krylov.chebyshev_apply(G, minv, e, degree, bound, 100.0) for e in np.eye(N)])
        assert np.linalg.norm(P - P.T) <= 1e-12 * np.linalg.norm(P)
        assert np.linalg.eigvalsh(0.5 * (P + P.T))[0] > 0.0
    # the positivity rests on the bound: an interval ending at half the largest
    # eigenvalue gives an indefinite polynomial
    P = np.column_stack([krylov.chebyshev_apply(G, minv, e, 4, 0.5 * lam[-1], 100.0) for e in np.eye(N)])
    assert np.linalg.eigvalsh(0.5 * (P + P.T))[0] < 0.0


def test_degree_one_takes_the_jacobi_iterates():
    G, S = hybrid_system("cfg2", 10)
    minv = krylov.jacobi(G)
    for k in (4, 25):
        x1, it1, _ = krylov.pcg(G, S, minv, rtol=0.0, maxit=k)
        x2, it2, _ = krylov.chebyshev_pcg(G, S, minv, 1, 100.0, rtol=0.0, maxit=k)
        assert it1 == it2 == k
        assert np.linalg.norm(x1 - x2) <= 1e-10 * np.linalg.norm(x1)


@pytest.mark.parametrize("name,n,degree", [("cfg2", 16, 4), ("cfg2", 16, 8), ("cfg3", 3, 4)])
def test_reaches_the_direct_solution(name, n, degree):
    G, S = hybrid_system(name, n)
    minv = krylov.jacobi(G)
    ref = spla.spsolve(G.tocsc(), S)
    x, it, hist = krylov.chebyshev_pcg(G, S, minv, degree, 100.0, rtol=1e-13)
    assert hist[-1] <= 1e-13
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
    _, it_j, _ = krylov.pcg(G, S, minv, rtol=1e-13)
    assert it < it_j   # fewer CG iterations (each applies G `degree` times)


def bf16_round(x):
    """Round to the nearest BF16 value (8 significant bits), ties to even: the values
    the reduced-precision Chebyshev steps read."""
    x = np.asarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("name,n,degree,ratio", [("cfg2", 6, 24, 10000.0), ("cfg3", 2, 24, 3000.0),
                                                 ("cfg2", 6, 4, 1000.0)])
def test_polynomial_of_the_bf16_matrix_stays_spd(name, n, degree, ratio):
    """The steps may use G~ = bf16(G) (symmetric, since equal entries round alike) under
    the Gershgorin bound of the exact M^{-1} G: the preconditioner p(M^{-1} G~) M^{-1} is
    still symmetric positive definite (the residual polynomial keeps p > 0 a little below
    0, where rounding may push small eigenvalues of G~), at the bench's degrees and
    ratios; and CG with it reaches the FP64 solution of G W = S."""
    G, S = hybrid_system(name, n)
    Gt = G.copy()
    Gt.data = bf16_round(Gt.data)
    assert abs(Gt - Gt.T).max() == 0.0
    minv = krylov.jacobi(G)
    bound = krylov.gershgorin_bound(G, minv)
    N = G.shape[0]
    P = np.column_stack([krylov.chebyshev_apply(Gt, minv, e, degree, bound, ratio) for e in np.eye(N)])
    assert np.linalg.norm(P - P.T) <= 1e-10 * np.linalg.norm(P)
    assert np.linalg.eigvalsh(0.5 * (P + P.T))[0] > 0.0
    ref = spla.spsolve(G.tocsc(), S)
    x = np.zeros(N)
    r = S.copy()
    z = P @ r
    p = z.copy()
    rz = r @ z
    for it in range(2000):
        q = G @ p
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        if np.linalg.norm(r) <= 1e-12 * np.linalg.norm(S):
            break
        z = P @ r
        rzn = r @ z
        p = z + (rzn / rz) * p
        rz = rzn
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
