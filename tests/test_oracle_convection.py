"""Pins for the oracle's co-volume convection form b_h (Section 2, item 6; Eq. 9).

* The flux F_{sigma sigma'} is checked against a brute-force construction of
  the co-volume interface tau_{sigma sigma'}: its area normal from the
  vertices, its centroid, and the affine CR velocity evaluated there.
* The two forms of b_h printed in the paper agree.
* The identity sum_{sigma'} F = -U_sigma . a_sigma when sum U . a = 0, and
  b_h(u, u) = 0 when div_h u = 0.
* The Newton derivative equals central differences (exact for a quadratic),
  and the Oseen matrix applied to w gives c(w).
"""

import numpy as np
import pytest

import synth
from oracle import convection, elements, pipeline, topology
from oracle.coupled import assemble, element_blocks

RNG = np.random.default_rng(99)


def random_simplices(d, count=40):
    X = RNG.normal(size=(count, d + 1, d))
    det = np.linalg.det(X[:, 1:] - X[:, :1])
    return X[np.abs(det) > 0.05]


def geom_of(X):
    ne, dp1, d = X.shape
    return elements.geometry(X.reshape(-1, d), np.arange(ne * dp1).reshape(ne, dp1))


def cr_value(X, U, x):
    """u_K(x) = sum_l U_l phi_l(x), phi_l = 1 - d lambda_l (barycentric form)."""
    ne, dp1, d = X.shape
    M = np.concatenate([np.transpose(X, (0, 2, 1)), np.ones((ne, 1, dp1))], axis=1)
    lam = np.linalg.solve(M, np.concatenate([x, np.ones((ne, 1))], axis=1)[..., None])[..., 0]
    phi = 1.0 - d * lam
    return np.einsum("kl,kld->kd", phi, U)


@pytest.mark.parametrize("d", [2, 3])
def test_flux_matches_covolume_interface(d):
    X = random_simplices(d)
    g = geom_of(X)
    U = RNG.normal(size=X.shape)
    F = convection.fluxes(U, g["a"])
    xK = X.mean(axis=1)
    for l in range(d + 1):
        for m in range(d + 1):
            if l == m:
                continue
            # tau_{lm}: the common part of the two co-volumes, spanned by x_K and
            # the vertices shared by faces l and m (all but vertices l and m)
            shared = [v for v in range(d + 1) if v not in (l, m)]
            P = [xK] + [X[:, v] for v in shared]
            if d == 2:
                t = P[1] - P[0]
                nvec = np.stack([t[:, 1], -t[:, 0]], axis=1)
                cen = 0.5 * (P[0] + P[1])
            else:
                nvec = 0.5 * np.cross(P[1] - P[0], P[2] - P[0])
                cen = (P[0] + P[1] + P[2]) / 3.0
            # orient from D_{K,l} to D_{K,m}: towards the centroid of the cone
            # D_{K,m} (base: face m, apex: x_K)
            cm = (xK + X.sum(axis=1) - X[:, m]) / (d + 1)
            sgn = np.sign(np.einsum("kd,kd->k", cm - cen, nvec))
            nvec = nvec * sgn[:, None]
            # the paper's closed forms for the area normal and the centroid
            assert np.allclose(nvec, (g["a"][:, m] - g["a"][:, l]) / (d + 1), rtol=1e-10, atol=1e-12)
            assert np.allclose(cen, g["xs"][:, l] + g["xs"][:, m] - xK, rtol=1e-12, atol=1e-12)
            flux = np.einsum("kd,kd->k", cr_value(X, U, cen), nvec)
            assert np.allclose(F[:, l, m], flux, rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("d", [2, 3])
def test_two_forms_of_bh_agree(d):
    X = random_simplices(d)
    g = geom_of(X)
    U, V = RNG.normal(size=X.shape), RNG.normal(size=X.shape)
    pairs = convection.bh_pairs(U, V, g["a"])
    c = convection.element_convection(U, g["a"])
    assert np.isclose(pairs, np.einsum("kld,kld->", V, c), rtol=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_flux_sum_identity(d):
    X = random_simplices(d)
    g = geom_of(X)
    a = g["a"]
    U = RNG.normal(size=X.shape)
    # remove the element divergence: U -= t a with t = sum U.a / sum a.a
    t = np.einsum("kld,kld->k", U, a) / np.einsum("kld,kld->k", a, a)
    U = U - t[:, None, None] * a
    F = convection.fluxes(U, a)
    assert np.allclose(F, -np.transpose(F, (0, 2, 1)), atol=1e-12)
    lhs = F.sum(axis=2)                      # F_{ll} = 0
    assert np.allclose(lhs, -np.einsum("kld,kld->kl", U, a), rtol=1e-10, atol=1e-11)


@pytest.mark.parametrize("dim", [2, 3])
def test_bh_vanishes_on_discretely_divergence_free_fields(dim):
    if dim == 2:
        coords, elems = synth.mesh2d_square(5, 0.2, 4)
    else:
        coords, elems = synth.mesh3d_kuhn(2)
    modes = synth.fourier_modes(dim, 5)
    fbar = synth.element_means(lambda x: synth.fourier_force(x, modes), coords, elems, order=2)
    ref = pipeline.direct(coords, elems, 1.0, 10.0, fbar, dense=True)
    Ul = convection.gather_local(ref["U"], ref["topo"])
    val = convection.bh_pairs(Ul, Ul, ref["geom"]["a"])
    scale = np.abs(Ul).max() ** 3 * np.abs(ref["geom"]["a"]).max() * elems.shape[0]
    assert abs(val) < 1e-13 * scale
    # and it does not vanish for a field that is not divergence free
    R = RNG.normal(size=Ul.shape) * (ref["topo"]["elem_face"] >= 0)[:, :, None]
    assert abs(convection.bh_pairs(R, R, ref["geom"]["a"])) > 1e-6


@pytest.mark.parametrize("d", [2, 3])
def test_newton_jacobian_is_exact_derivative(d):
    X = random_simplices(d, 20)
    g = geom_of(X)
    W = RNG.normal(size=X.shape)
    J = convection.newton_jacobian(W, g["a"])
    ne, dp1, _ = X.shape
    Jfd = np.zeros_like(J)
    for col in range(dp1 * d):
        E = np.zeros((dp1 * d,))
        E[col] = 1.0
        E = E.reshape(dp1, d)
        cp = convection.element_convection(W + E, g["a"]).reshape(ne, -1)
        cm = convection.element_convection(W - E, g["a"]).reshape(ne, -1)
        Jfd[:, :, col] = 0.5 * (cp - cm)      # exact for a quadratic
    assert np.allclose(J, Jfd, rtol=1e-11, atol=1e-11)
    c = convection.element_convection(W, g["a"]).reshape(ne, -1)
    assert np.allclose(np.einsum("kab,kb->ka", J, W.reshape(ne, -1)), 2 * c, rtol=1e-11, atol=1e-11)
    N = convection.oseen_matrix(W, g["a"])
    assert np.allclose(np.einsum("kab,kb->ka", N, W.reshape(ne, -1)), c, rtol=1e-11, atol=1e-11)


def test_newton_step_converges_quadratically():
    """Repeated Newton steps on the coupled system drive the NS residual down."""
    coords, elems = synth.mesh2d_square(6, 0.1, 8)
    modes = synth.fourier_modes(2, 2)
    fbar = 5.0 * synth.element_means(lambda x: synth.fourier_force(x, modes), coords, elems, order=3)
    t = topology.build_faces(elems)
    w = np.zeros((t["nf"], 2))
    res = []
    for _ in range(6):
        sol = pipeline.direct(coords, elems, 0.05, 0.0, fbar, "newton", w)
        Ul = convection.gather_local(sol["U"], sol["topo"])
        c = convection.element_convection(Ul, sol["geom"]["a"])
        A_K, D_K, R_K = element_blocks(sol["topo"], sol["geom"], 0.05, 0.0, fbar)
        A, D, R = assemble(sol["topo"], A_K, D_K, R_K)
        cg = np.zeros(t["nf"] * 2)
        dofs = elements.local_dofs(t)
        cflat = c.reshape(c.shape[0], -1)
        np.add.at(cg, dofs[dofs >= 0], cflat[dofs >= 0])
        F = A @ sol["U"].ravel() + cg + D.T @ np.delete(sol["P"], 0) - R
        res.append(np.linalg.norm(F) / np.linalg.norm(R))
        w = sol["U"]
    assert res[-1] < 1e-13
    for k in range(1, 3):                    # quadratic: e_{k+1} <= C e_k^2
        assert res[k + 1] <= 5.0 * res[k] ** 2
