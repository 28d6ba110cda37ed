"""Pins for the oracle's geometry and element matrices (Section 2; Section 3.1).

Each check compares the oracle against an independent construction: the
barycentric-coordinate form of the CR basis, closed-form simplex integrals,
and direct quadrature of the Raviart-Thomas reconstruction.
"""

import math

import numpy as np
import pytest

import synth
from oracle import elements

RNG = np.random.default_rng(1234)


def random_simplices(d, count=50):
    X = RNG.normal(size=(count, d + 1, d))
    J = X[:, 1:] - X[:, :1]
    det = np.linalg.det(J)
    X = X[np.abs(det) > 0.05]
    return X


def as_mesh(X):
    ne, dp1, d = X.shape
    coords = X.reshape(-1, d)
    elems = np.arange(ne * dp1, dtype=np.int32).reshape(ne, dp1)
    return coords, elems


def barycentric_gradients(X):
    """grad lambda_v for each vertex v: rows of the inverse of [[x_v]; [1]]."""
    ne, dp1, d = X.shape
    M = np.concatenate([np.transpose(X, (0, 2, 1)), np.ones((ne, 1, dp1))], axis=1)
    Minv = np.linalg.inv(M)            # lambda = Minv @ [x; 1]
    return Minv[:, :, :d]              # [ne, vertex, d]


@pytest.mark.parametrize("d", [2, 3])
def test_volume_and_closure(d):
    X = random_simplices(d)
    g = elements.geometry(*as_mesh(X))
    J = X[:, 1:] - X[:, :1]
    vol = np.abs(np.linalg.det(J)) / math.factorial(d)
    assert np.allclose(g["vol"], vol, rtol=1e-13)
    # sum of |sigma| n_sigma over the faces of a closed simplex is zero
    assert np.abs(g["a"].sum(axis=1)).max() < 1e-12 * np.abs(g["a"]).max()


@pytest.mark.parametrize("d", [2, 3])
def test_area_normal_is_barycentric_gradient(d):
    """a_{K,sigma} = -d |K| grad(lambda_{s_sigma}), s_sigma opposite sigma."""
    X = random_simplices(d)
    g = elements.geometry(*as_mesh(X))
    gl = barycentric_gradients(X)
    expect = -d * g["vol"][:, None, None] * gl
    assert np.allclose(g["a"], expect, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_cr_gradients_closed_form(d):
    """phi_sigma = 1 - d lambda_{s_sigma}, so grad phi_sigma = -d grad lambda."""
    X = random_simplices(d)
    g = elements.geometry(*as_mesh(X))
    gphi = elements.cr_gradients(g)
    expect = -d * barycentric_gradients(X)
    assert np.allclose(gphi, expect, rtol=1e-10, atol=1e-10)


def simplex_monomial(d, alpha):
    """(1/|K|) int_K prod lambda^alpha = d! prod alpha! / (|alpha| + d)!."""
    return math.factorial(d) * np.prod([math.factorial(a) for a in alpha]) / math.factorial(sum(alpha) + d)


@pytest.mark.parametrize("d", [2, 3])
def test_S_matches_closed_form_integrals(d):
    """S_K = nu int grad phi . grad phi' + mu (lumped mass |K|/(d+1) delta)."""
    X = random_simplices(d)
    g = elements.geometry(*as_mesh(X))
    nu, mu = 0.7, 3.0
    S = elements.local_S(g, nu, mu)
    gphi = -d * barycentric_gradients(X)
    stiff = nu * g["vol"][:, None, None] * np.einsum("kad,kbd->kab", gphi, gphi)
    mass = mu * g["vol"][:, None, None] / (d + 1) * np.eye(d + 1)
    assert np.allclose(S, stiff + mass, rtol=1e-11, atol=1e-12)


def test_2d_cr_mass_is_diagonal_and_equals_lumped():
    """In 2D the exact CR mass int phi phi' is |K|/3 delta (Section 2, item 3)."""
    d = 2
    # int (1 - 2 l_a)(1 - 2 l_b) / |K| = 1 - 2E[l_a] - 2E[l_b] + 4E[l_a l_b]
    for a in range(3):
        for b in range(3):
            alpha = [0, 0, 0]
            alpha[a] += 1
            alpha[b] += 1
            val = 1 - 2 * simplex_monomial(d, [1, 0, 0]) * 2 + 4 * simplex_monomial(d, alpha)
            assert abs(val - (1 / 3 if a == b else 0.0)) < 1e-15


@pytest.mark.parametrize("d", [2, 3])
def test_R_is_rt_reconstruction_of_constant_source(d):
    """(R_K)_{i,sigma} = n^(i) int_K f . psi_{K,sigma} for constant f (Eq. 8).

    psi_{K,sigma}(x) = |sigma|/(d|K|) (x - s_sigma) is affine, so the
    one-point centroid rule integrates it exactly.
    """
    X = random_simplices(d)
    g = elements.geometry(*as_mesh(X))
    f = RNG.normal(size=(X.shape[0], d))
    R = elements.local_R(g, f).reshape(X.shape[0], d + 1, d)
    area = np.linalg.norm(g["a"], axis=2)
    n = g["a"] / area[:, :, None]
    xK = X.mean(axis=1)
    for l in range(d + 1):
        psi_mean = area[:, l, None] / (d * g["vol"][:, None]) * (xK - X[:, l])
        integral = g["vol"] * np.einsum("kd,kd->k", f, psi_mean)
        expect = n[:, l] * integral[:, None]
        assert np.allclose(R[:, l], expect, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_element_means_exact_for_quadratics(d):
    """The shared generator's element means are exact for quadratic sources."""
    if d == 2:
        coords, elems = synth.mesh2d_square(3, perturb=0.2, seed=5)
    else:
        coords, elems = synth.mesh3d_kuhn(2)
    X = coords[elems]
    c = RNG.normal(size=(d, d))

    def f(x):
        return np.stack([(x[:, 0] ** 2) * c[i, 0] + x[:, 1] * x[:, -1] * c[i, 1] for i in range(d)], axis=1)

    got = synth.element_means(f, coords, elems, order=3)
    # closed form: x_a x_b = sum_{u,v} X_ua X_vb lambda_u lambda_v
    E2 = np.full((d + 1, d + 1), simplex_monomial(d, [1, 1] + [0] * (d - 1)))
    np.fill_diagonal(E2, simplex_monomial(d, [2] + [0] * d))
    m00 = np.einsum("kua,kvb,uv->k", X[..., :1], X[..., :1], E2)
    m1e = np.einsum("kua,kvb,uv->k", X[..., 1:2], X[..., -1:], E2)
    expect = np.stack([m00 * c[i, 0] + m1e * c[i, 1] for i in range(d)], axis=1)
    assert np.allclose(got, expect, rtol=1e-12, atol=1e-13)


def test_generated_meshes():
    coords, elems = synth.mesh2d_square(8, perturb=0.2, seed=0)
    assert elems.shape == (128, 3) and coords.shape == (81, 2)
    X = coords[elems]
    J = X[:, 1:] - X[:, :1]
    assert np.all(np.linalg.det(J) > 0)
    assert np.isclose(np.abs(np.linalg.det(J)).sum() / 2, 1.0)
    coords, elems = synth.mesh3d_kuhn(3)
    X = coords[elems]
    vol = np.abs(np.linalg.det(X[:, 1:] - X[:, :1])) / 6
    assert elems.shape == (162, 4) and np.isclose(vol.sum(), 1.0) and vol.min() > 0
