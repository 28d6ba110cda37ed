"""Pins for the oracle's hybridisation (Section 3.2) against the coupled system.

The hybrid method reaches the coupled solution exactly (Section 3.2, item 2),
so its U and P are compared with a library direct solve of Eq. 10 on small
meshes, for transient Stokes, steady Stokes (mu = 0, E_K from the maximal
independent set) and a Newton step.  Further pins: D U = 0 element by
element, equal doubled velocities (Eq. 15), G symmetric positive definite
for mu > 0 (item 6), symmetric for steady Stokes, the stencil of A
(item 5), invariance under the choice of K_0, and the constant-source
closed form (Section 4.1: U = 0 and the exact pressure).
"""

import numpy as np
import pytest

import synth
from oracle import coupled, elements, hybrid, pipeline

RNG = np.random.default_rng(7)


def small_case(dim, n, perturb=0.2, seed=3):
    if dim == 2:
        coords, elems = synth.mesh2d_square(n, perturb=perturb, seed=seed)
    else:
        coords, elems = synth.mesh3d_kuhn(n)
    modes = synth.fourier_modes(dim, 11)
    fbar = synth.element_means(lambda x: synth.fourier_force(x, modes), coords, elems, order=3)
    return coords, elems, fbar


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def face_velocity(coords, elems, seed=3):
    from oracle import topology
    t = topology.build_faces(elems)
    xs = coords[t["face_vertices"]].mean(axis=1)
    return synth.stream_velocity(xs, seed=seed)


CASES = [
    (2, 4, 1.0, 100.0, "none"),
    (2, 6, 1.0, 1000.0, "none"),
    (3, 2, 1.0, 1000.0, "none"),
    (2, 5, 1.0, 0.0, "none"),
    (3, 2, 1.0, 0.0, "none"),
    (2, 5, 0.01, 0.0, "newton"),
    (2, 5, 0.01, 0.0, "oseen"),
    (2, 4, 0.05, 10.0, "newton"),
]


@pytest.mark.parametrize("dim,n,nu,mu,conv", CASES)
def test_hybrid_equals_coupled(dim, n, nu, mu, conv):
    coords, elems, fbar = small_case(dim, n)
    w = face_velocity(coords, elems) if conv != "none" else None
    ref = pipeline.direct(coords, elems, nu, mu, fbar, conv, w, dense=True)
    hyb = pipeline.hybrid(coords, elems, nu, mu, fbar, conv, w, method="direct")
    vol = ref["geom"]["vol"]
    assert rel(hyb["U"], ref["U"]) < 1e-10
    assert rel(coupled.normalise_pressure(hyb["P"], vol),
               coupled.normalise_pressure(ref["P"], vol)) < 1e-9
    assert hyb["stats"]["jump"] < 1e-10 * max(np.abs(hyb["U"]).max(), 1e-300)
    # the recovered pair satisfies the coupled equations
    assert coupled.coupled_residual(ref["A"], ref["D"], ref["R"], hyb["U"].ravel(), hyb["P"]) < 1e-10


@pytest.mark.parametrize("dim", [2, 3])
def test_discrete_divergence_vanishes_per_element(dim):
    coords, elems, fbar = small_case(dim, 4 if dim == 2 else 2)
    hyb = pipeline.hybrid(coords, elems, 1.0, 100.0, fbar, method="pcg", rtol=1e-14)
    g, t = hyb["geom"], hyb["topo"]
    U = hyb["U"]
    Ul = np.where((t["elem_face"] >= 0)[:, :, None], U[np.maximum(t["elem_face"], 0)], 0.0)
    div = np.einsum("kld,kld->k", Ul, g["a"])          # int_K div u = sum U . a  (incl. K_0)
    scale = np.abs(g["a"]).max() * np.abs(U).max()
    assert np.abs(div).max() < 1e-11 * scale


@pytest.mark.parametrize("dim,n", [(2, 2), (2, 4), (2, 8), (3, 1), (3, 2)])
def test_G_symmetric_positive_definite(dim, n):
    coords, elems, fbar = small_case(dim, n)
    topo, geom, A_K, D_K, R_K = pipeline.setup(coords, elems, 1.0, 100.0, fbar)
    h = hybrid.hybridise(topo, A_K, D_K, R_K, 100.0)
    G = h["G"].toarray()
    assert np.abs(G - G.T).max() <= 1e-13 * np.abs(G).max()
    ev = np.linalg.eigvalsh(0.5 * (G + G.T))
    assert ev.min() > 0


def test_G_steady_stokes_symmetric_indefinite():
    coords, elems, fbar = small_case(2, 4)
    topo, geom, A_K, D_K, R_K = pipeline.setup(coords, elems, 1.0, 0.0, fbar)
    h = hybrid.hybridise(topo, A_K, D_K, R_K, 0.0)
    G = h["G"].toarray()
    assert np.abs(G - G.T).max() <= 1e-12 * np.abs(G).max()
    ev = np.linalg.eigvalsh(0.5 * (G + G.T))
    assert ev.min() < 0 < ev.max()
    assert np.abs(ev).min() > 1e-12 * np.abs(ev).max()      # invertible
    # E_K + E_L = 0 on every interior face (Eq. 11)
    E, fe, fl, d = h["E"], topo["face_elems"], topo["face_local"], topo["d"]
    for f in range(topo["nf"]):
        K, L = fe[f]
        assert np.all(E[K, fl[f, 0] * d:(fl[f, 0] + 1) * d] + E[L, fl[f, 1] * d:(fl[f, 1] + 1) * d] == 0)


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 2)])
def test_G_has_the_stencil_of_A(dim, n):
    coords, elems, fbar = small_case(dim, n)
    topo, geom, A_K, D_K, R_K = pipeline.setup(coords, elems, 1.0, 100.0, fbar)
    h = hybrid.hybridise(topo, A_K, D_K, R_K, 100.0)
    d = topo["d"]
    s = (topo["elem_face"] >= 0).sum(axis=1)
    nblocks = int((s * (s - 1)).sum()) + topo["nf"]
    G = h["G"].tocoo()
    blocks = {(r // d, c // d) for r, c, v in zip(G.row, G.col, G.data) if v != 0.0}
    assert len(blocks) == nblocks
    A, D, R = coupled.assemble(topo, A_K, D_K, R_K)
    A = A.tocoo()
    ablocks = {(r // d, c // d) for r, c in zip(A.row, A.col)}
    assert blocks == ablocks
    # every d x d block is full: the components couple (Section 1)
    assert G.nnz == nblocks * d * d


def test_B_bound():
    """|B_K| >= lambda_min(Â_K^{-1}) ||D_K||^2 > 0 (Section 3.2, item 3)."""
    coords, elems, fbar = small_case(2, 4)
    topo, geom, A_K, D_K, R_K = pipeline.setup(coords, elems, 1.0, 100.0, fbar)
    h = hybrid.hybridise(topo, A_K, D_K, R_K, 100.0)
    mask = elements.interior_mask(topo)
    for K in range(topo["ne"]):
        idx = np.flatnonzero(mask[K])
        Ainv = h["Ainv"][K][np.ix_(idx, idx)]
        lam = np.linalg.eigvalsh(Ainv).min()
        assert h["B"][K] >= lam * np.dot(D_K[K], D_K[K]) * (1 - 1e-12) > 0


@pytest.mark.parametrize("dim", [2, 3])
def test_k0_invariance(dim):
    coords, elems, fbar = small_case(dim, 4 if dim == 2 else 2)
    a = pipeline.hybrid(coords, elems, 1.0, 100.0, fbar, method="direct", k0=0)
    b = pipeline.hybrid(coords, elems, 1.0, 100.0, fbar, method="direct", k0=elems.shape[0] - 1)
    vol = a["geom"]["vol"]
    assert rel(a["U"], b["U"]) < 1e-11
    assert rel(coupled.normalise_pressure(a["P"], vol), coupled.normalise_pressure(b["P"], vol)) < 1e-10
    assert a["P"][0] == 0.0 and b["P"][-1] == 0.0


@pytest.mark.parametrize("dim,mu", [(2, 100.0), (3, 1000.0), (2, 0.0)])
def test_constant_source_gives_zero_velocity_and_exact_pressure(dim, mu):
    """Section 4.1: constant f gives U = 0 and P_K - P_{K_0} = f . (x_K - x_{K_0})."""
    coords, elems, _ = small_case(dim, 5 if dim == 2 else 2)
    c = np.array([0.7, -1.3, 0.4][:dim])
    fbar = np.tile(c, (elems.shape[0], 1))
    h = pipeline.hybrid(coords, elems, 1.0, mu, fbar, method="direct")
    xK = h["geom"]["xK"]
    assert np.abs(h["U"]).max() < 1e-12
    assert np.abs(h["P"] - (xK - xK[0]) @ c).max() < 1e-12


def test_multiple_right_hand_sides():
    coords, elems, fbar = small_case(2, 4)
    fb2 = np.stack([fbar, 2.0 * fbar + 1.0])
    topo, geom, A_K, D_K, R_K = pipeline.setup(coords, elems, 1.0, 100.0, fbar)
    R2 = np.stack([elements.local_R(geom, f) * elements.interior_mask(topo) for f in fb2])
    h = hybrid.hybridise(topo, A_K, D_K, R2, 100.0)
    h1 = hybrid.hybridise(topo, A_K, D_K, R2[1], 100.0)
    assert np.allclose(h["S"][1], h1["S"], rtol=1e-14, atol=0)
