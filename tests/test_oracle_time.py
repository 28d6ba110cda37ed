"""Pins for the oracle's implicit Euler step (mu = 1/dt; Section 2 with the
lumped mass of Section 3.1 applied to the previous time level).

* The previous-level term, assembled over the mesh, is mu M u^n with M the
  lumped mass: per face the sum of |K|/(d+1) over its two simplices, counted
  here by a plain loop over simplices and faces.
* The steady solution (mu = 0) is a fixed point of a time step: with u^n equal
  to it the step returns it, because the mass term of S_K and of R_K cancel
  exactly when they agree.
* The step is first-order accurate in time: on a fixed mesh the differences of
  successive halvings of dt shrink by a factor of 2 (the spatial error is the
  same for every dt and cancels in the differences).
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import coupled, elements, hybrid, pipeline, topology


def case(dim, n, seed=5):
    if dim == 2:
        coords, elems = synth.mesh2d_square(n, perturb=0.2, seed=seed)
    else:
        coords, elems = synth.mesh3d_kuhn(n)
    modes = synth.fourier_modes(dim, 13)
    fbar = synth.element_means(lambda x: synth.fourier_force(x, modes), coords, elems, order=3)
    return coords, elems, fbar


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 2)])
def test_previous_level_term_is_the_lumped_mass(dim, n):
    coords, elems, fbar = case(dim, n)
    mu, nu = 37.0, 0.7
    topo = topology.build_faces(elems)
    geom = elements.geometry(coords, elems)
    u_prev = np.random.default_rng(3).standard_normal((topo["nf"], dim))
    _, _, R0 = coupled.element_blocks(topo, geom, nu, mu, fbar)
    _, _, R1 = coupled.element_blocks(topo, geom, nu, mu, fbar, u_prev=u_prev)
    _, _, Rg0 = coupled.assemble(topo, *coupled.element_blocks(topo, geom, nu, mu, fbar))
    _, _, Rg1 = coupled.assemble(topo, *coupled.element_blocks(topo, geom, nu, mu, fbar, u_prev=u_prev))
    # lumped mass by a plain loop: every interior face of every simplex gets |K|/(d+1)
    M = np.zeros(topo["nf"])
    for K in range(elems.shape[0]):
        for l in range(dim + 1):
            f = topo["elem_face"][K, l]
            if f >= 0:
                M[f] += geom["vol"][K] / (dim + 1)
    expect = (mu * M[:, None] * u_prev).ravel()
    assert np.abs((Rg1 - Rg0) - expect).max() <= 1e-13 * np.abs(expect).max()
    # exterior unknowns carry nothing
    ext = ~elements.interior_mask(topo)
    assert np.all((R1 - R0)[ext] == 0.0)


@pytest.mark.parametrize("dim,n", [(2, 7), (3, 2)])
def test_steady_solution_is_a_fixed_point_of_the_time_step(dim, n):
    coords, elems, fbar = case(dim, n)
    nu, mu = 1.3, 250.0
    steady = pipeline.direct(coords, elems, nu, 0.0, fbar, dense=True)
    step = pipeline.direct(coords, elems, nu, mu, fbar, dense=True, u_prev=steady["U"])
    vol = steady["geom"]["vol"]
    assert np.linalg.norm(step["U"] - steady["U"]) <= 1e-11 * np.linalg.norm(steady["U"])
    Ps = coupled.normalise_pressure(steady["P"], vol)
    assert np.linalg.norm(coupled.normalise_pressure(step["P"], vol) - Ps) <= 1e-10 * np.linalg.norm(Ps)
    # a different previous level moves the solution (the term is not silently dropped)
    other = pipeline.direct(coords, elems, nu, mu, fbar, dense=True, u_prev=np.zeros_like(steady["U"]))
    assert np.linalg.norm(other["U"] - steady["U"]) > 1e-3 * np.linalg.norm(steady["U"])


def test_hybrid_step_equals_the_coupled_step():
    """The hybridised step (G, S from R_K with the previous level, recovery with
    the same R_K) reaches the coupled step exactly (Section 3.2, item 2)."""
    coords, elems, fbar = case(2, 6)
    nu, mu = 1.0, 100.0
    topo = topology.build_faces(elems)
    u_prev = np.random.default_rng(9).standard_normal((topo["nf"], 2))
    ref = pipeline.direct(coords, elems, nu, mu, fbar, dense=True, u_prev=u_prev)
    topo, geom, A_K, D_K, R_K = pipeline.setup(coords, elems, nu, mu, fbar, u_prev=u_prev)
    h = hybrid.hybridise(topo, A_K, D_K, R_K, mu)
    W = spla.spsolve(h["G"].tocsc(), h["S"])
    U, P, _ = hybrid.recover(h, topo, W, R_K)
    assert np.linalg.norm(U.ravel() - ref["U"].ravel()) <= 1e-11 * np.linalg.norm(ref["U"])
    vol = geom["vol"]
    Pr = coupled.normalise_pressure(ref["P"], vol)
    assert np.linalg.norm(coupled.normalise_pressure(P, vol) - Pr) <= 1e-10 * np.linalg.norm(Pr)


def test_implicit_euler_is_first_order_in_time():
    """u(x, t) = exp(-t) u0(x) with u0 = curl(sin^2 pi x sin^2 pi y), p = 0,
    f = du/dt - nu Lap u = exp(-t) (-u0 - nu Lap u0), integrated to T = 0.2."""
    n, nu, T = 10, 1.0, 0.2
    coords, elems = synth.mesh2d_square(n)
    topo = topology.build_faces(elems)
    ms = synth.manufactured_stokes(2, mu=-1.0, nu=nu)           # f0 = -u0 - nu Lap u0
    f0 = synth.element_means(ms["f"], coords, elems, order=4)
    xs = coords[topo["face_vertices"]].mean(axis=1)
    u0 = ms["u"](xs)

    def run(steps):
        dt = T / steps
        u = u0.copy()
        for k in range(1, steps + 1):
            out = pipeline.direct(coords, elems, nu, 1.0 / dt, np.exp(-k * dt) * f0, dense=True, u_prev=u)
            u = out["U"].reshape(-1, 2)
        return u

    u4, u8, u16 = run(4), run(8), run(16)
    ratio = np.linalg.norm(u4 - u8) / np.linalg.norm(u8 - u16)
    assert 1.8 <= ratio <= 2.2
    # and the discrete solution follows the decay of the exact one, within the
    # spatial error of the 10 x 10 mesh (about 6% at the face centroids)
    assert np.linalg.norm(u16 - np.exp(-T) * u0) <= 0.08 * np.linalg.norm(np.exp(-T) * u0)
    assert np.linalg.norm(u16 - u0) >= 0.15 * np.linalg.norm(u0)
