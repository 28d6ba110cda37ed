"""The host eigensolver of the Lanczos matrix (csrc/tridiag.h, no GPU).

cr_deflation_lanczos and cr_solve_ritz take their Ritz vectors from the k
smallest eigenpairs of the symmetric tridiagonal Lanczos matrix T, which the
library computes on the host by bisection on Sturm counts and inverse
iteration.  This test compiles that header with the host compiler and checks it
against NumPy's dense symmetric eigensolver: the eigenvalues, and eigenvectors
that are orthonormal with small residuals ||T s - theta s||.  The cases cover
a random matrix, a Lanczos matrix of CG on the oracle's G (widely spread
eigenvalues), clustered eigenvalues, an exactly repeated eigenvalue (a
decoupled matrix: zero off-diagonal), and k larger than the matrix.
"""

import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r"""
#include <cstdio>
#include <vector>
#include "tridiag.h"
int main() {
    int n, k;
    if (std::scanf("%d %d", &n, &k) != 2) return 2;
    std::vector<double> a(n), b(n > 1 ? n - 1 : 0), th, S;
    for (auto& v : a) std::scanf("%lf", &v);
    for (auto& v : b) std::scanf("%lf", &v);
    crhyb::tridiag_smallest_eigen(a, b, k, th, S);
    std::printf("%zu\n", th.size());
    for (double t : th) std::printf("%.17g\n", t);
    for (double s : S) std::printf("%.17g\n", s);
    return 0;
}
"""


@pytest.fixture(scope="module")
def solver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("tridiag")
    src, exe = d / "t.cpp", d / "t"
    src.write_text(SRC)
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_2101_03777_gb300", "csrc"), str(src),
                    "-o", str(exe)], check=True)

    def run(a, b, k):
        inp = f"{len(a)} {k}\n" + " ".join(repr(float(x)) for x in a) + "\n" + " ".join(repr(float(x)) for x in b)
        out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout.split()
        kk = int(out[0])
        th = np.array([float(x) for x in out[1:1 + kk]])
        S = np.array([float(x) for x in out[1 + kk:]]).reshape(len(a), kk)
        return th, S
    return run


def dense(a, b):
    return np.diag(a) + np.diag(b, 1) + np.diag(b, -1)


def check(run, a, b, k, vec_tol=1e-8):
    a, b = np.asarray(a, float), np.asarray(b, float)
    T = dense(a, b)
    ev = np.linalg.eigvalsh(T)
    th, S = run(a, b, k)
    kk = min(k, len(a))
    scale = np.abs(ev).max()
    assert th.shape == (kk,) and S.shape == (len(a), kk)
    assert np.allclose(th, ev[:kk], rtol=1e-12, atol=1e-13 * scale), (th, ev[:kk])
    assert np.abs(S.T @ S - np.eye(kk)).max() <= vec_tol
    for j in range(kk):
        assert np.linalg.norm(T @ S[:, j] - th[j] * S[:, j]) <= vec_tol * scale, j
    return th, S


def test_random_tridiagonal(solver):
    rng = np.random.default_rng(1)
    check(solver, rng.uniform(1, 5, 60), rng.uniform(-1, 1, 59), 8)


def test_lanczos_matrix_of_the_oracle(solver):
    """T of 80 Jacobi-PCG steps on the oracle's hybridised G (the matrix the library
    sees): its smallest eigenvalues span orders of magnitude."""
    import synth
    from oracle import hybrid, krylov, pipeline
    p = synth.config_problem("cfg2", n=12)
    topo, geom, A_K, D_K, R_K = pipeline.setup(p["coords"], p["elems"], p["nu"], p["mu"], p["fbar"][0], p["conv"])
    h = hybrid.hybridise(topo, A_K, D_K, R_K, p["mu"])
    G = h["G"].tocsr()
    minv = krylov.jacobi(G)
    _, _, T = krylov.lanczos_ritz(G, h["S"], lambda r: minv * r, 80, 4)
    th, _ = check(solver, np.diag(T), np.diag(T, 1), 8)
    assert th[0] < 0.1 * th[-1]


def test_clustered_eigenvalues(solver):
    """Eigenvalues 1e-9 apart (a near-copy, as the loss of orthogonality of Lanczos
    produces): the vectors must still come out orthonormal."""
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    lam = np.concatenate([[1.0, 1.0 + 1e-9, 1.0 + 2e-9], np.linspace(2, 10, 27)])
    # tridiagonalise Q diag(lam) Q^t by Lanczos in exact-enough arithmetic (Householder via scipy)
    import scipy.linalg as sla
    H, _ = sla.hessenberg(Q @ np.diag(lam) @ Q.T, calc_q=True)
    a, b = np.diag(H), np.diag(H, 1)
    check(solver, a, b, 5, vec_tol=1e-6)


def test_repeated_eigenvalue_of_a_decoupled_matrix(solver):
    """A zero off-diagonal splits T into blocks with the same eigenvalue."""
    a = np.array([2.0, 3.0, 2.0, 3.0, 7.0])
    b = np.array([0.5, 0.0, 0.5, 0.0])
    check(solver, a, b, 4)


def test_more_pairs_than_the_matrix_has(solver):
    th, S = solver(np.array([4.0, 1.0, 3.0]), np.array([0.2, 0.1]), 8)
    assert len(th) == 3 and S.shape == (3, 3)
    assert np.allclose(th, np.linalg.eigvalsh(dense([4.0, 1.0, 3.0], [0.2, 0.1])), rtol=1e-12)
