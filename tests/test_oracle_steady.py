"""Pins for the oracle's steady solver (oracle/steady.py).

The steady problem is Eq. 10 with mu = 0, whose plain definition is the
direct solve of the coupled system (coupled.solve_direct).  The oracle solves
it by flexible GMRES preconditioned by transient hybridised solves; it is
pinned by:
  * the lumped face mass against a plain loop over simplices;
  * the preconditioner against a direct solve of the transient coupled system
    [A_0 + mu M, D^t; D 0] z = [v; 0] (the previous-level encoding of v and
    the recovery);
  * the flexible GMRES cycle against its definition, the minimal residual over
    x_0 + span(Z), computed by dense least squares;
  * the steady solution against the direct solve (Stokes and Newton, 2D and
    3D), and the mesh independence of the number of steps the eigenvalues
    lambda/(lambda + mu) predict;
  * the Newton loop for the steady Navier-Stokes problem by the residual of the
    nonlinear scheme at its end point (b_h from the pinned convection module)
    and by its quadratic convergence.
"""

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import coupled, pipeline, steady, topology


def problem(dim, n, conv="none", perturb=0.2):
    if dim == 2:
        coords, elems = synth.mesh2d_square(n, perturb, 5)
    else:
        coords, elems = synth.mesh3d_kuhn(n)
    modes = synth.fourier_modes(dim, 1)
    fbar = synth.element_means(lambda x: synth.fourier_force(x, modes), coords, elems, order=3)
    w = None
    if conv != "none":
        t = topology.build_faces(elems)
        w = synth.stream_velocity(coords[t["face_vertices"]].mean(axis=1), seed=3)
    return coords, elems, fbar, w


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dim", [2, 3])
def test_face_mass_matches_a_loop_over_simplices(dim):
    coords, elems, fbar, _ = problem(dim, 5 if dim == 2 else 2)
    topo, geom, *_ = pipeline.setup(coords, elems, 1.0, 1.0, fbar)
    m = np.zeros(topo["nf"])
    for K in range(elems.shape[0]):
        for l in range(dim + 1):
            f = topo["elem_face"][K, l]
            if f >= 0:
                m[f] += geom["vol"][K] / (dim + 1)
    assert np.allclose(steady.face_mass(topo, geom), m, rtol=1e-14, atol=0)


@pytest.mark.parametrize("dim,n,conv", [(2, 6, "none"), (2, 6, "oseen"), (3, 2, "none")])
def test_preconditioner_is_the_transient_coupled_solve(dim, n, conv):
    """z = K_mu^{-1} [v; g]: the hybrid method on the transient system, its
    right-hand side encoded as a previous level and a divergence g, against a
    direct solve (g = 0 and g random)."""
    coords, elems, fbar, w = problem(dim, n, conv)
    nu, mu = 0.5, 7.0
    pre = steady.TransientPreconditioner(coords, elems, nu, mu, conv, w)
    topo, geom, A_K, D_K, _ = pipeline.setup(coords, elems, nu, mu, np.zeros((elems.shape[0], dim)), conv, w)
    A, D, _ = coupled.assemble(topo, A_K, D_K, np.zeros_like(A_K[:, :, 0]), 0)
    # the previous level contributes no convection term: only the mass and the viscous
    # and convective operator of the step enter A
    rng = np.random.default_rng(3)
    v = rng.standard_normal(A.shape[0])
    K = coupled.saddle_matrix(A, D)
    for g in (np.zeros(D.shape[0]), rng.standard_normal(D.shape[0])):
        zu, zp = pre(v, np.insert(g, 0, 7.0))          # the entry of K_0 is not used
        ref = spla.spsolve(K.tocsc(), np.concatenate([v, g]))
        assert rel(zu, ref[:A.shape[0]]) <= 1e-10
        assert zp[0] == 0.0 and rel(zp[1:], ref[A.shape[0]:]) <= 1e-9


def test_fgmres_cycle_is_the_minimal_residual_over_span_Z():
    rng = np.random.default_rng(4)
    n = 40
    K = sp.random(n, n, density=0.3, random_state=5) + 4 * sp.eye(n)
    b = rng.standard_normal(n)
    Ms = [np.diag(1.0 + rng.random(n)) for _ in range(12)]
    calls = []

    def precond(v):   # a different preconditioner at every step (the flexible case)
        z = Ms[len(calls) % len(Ms)] @ v
        calls.append(z)
        return z

    for k in (3, 6, 9):
        calls.clear()
        x, steps, _ = steady.fgmres(lambda y: K @ y, precond, b, restart=k, rtol=0.0, maxit=k)
        Z = np.array(calls[:k]).T
        y, *_ = np.linalg.lstsq(K @ Z, b, rcond=None)
        assert steps == k
        assert np.linalg.norm(x - Z @ y) <= 1e-9 * np.linalg.norm(Z @ y)


@pytest.mark.parametrize("dim,n,nu,conv,mu_pre", [(2, 10, 1.0, "none", 30.0), (2, 10, 0.01, "newton", 1.0),
                                                  (2, 8, 0.05, "oseen", 3.0), (3, 2, 1.0, "none", 30.0)])
def test_steady_solution_equals_the_direct_solve(dim, n, nu, conv, mu_pre):
    coords, elems, fbar, w = problem(dim, n, conv)
    ref = pipeline.direct(coords, elems, nu, 0.0, fbar, conv, w)
    U, P, st = steady.solve_steady(coords, elems, nu, fbar, conv, w, mu_pre=mu_pre, pre_conv="none", restart=60,
                                   rtol=1e-12)
    vol = ref["geom"]["vol"]
    assert st["relres"] <= 1e-11
    assert rel(U, ref["U"].ravel()) <= 1e-9
    assert rel(coupled.normalise_pressure(P, vol), coupled.normalise_pressure(ref["P"], vol)) <= 1e-9


def test_number_of_steps_does_not_grow_with_the_mesh():
    steps = []
    for n in (8, 16, 32):
        coords, elems, fbar, w = problem(2, n)
        _, _, st = steady.solve_steady(coords, elems, 1.0, fbar, mu_pre=30.0, restart=60, rtol=1e-10)
        steps.append(st["steps"])
    assert max(steps) - min(steps) <= 2 and max(steps) <= 15, steps


def test_newton_converges_quadratically_to_the_navier_stokes_solution():
    """The oracle's Newton loop (nu = 0.02, the seeded Fourier source; max |U| about
    0.76) ends at a solution of the nonlinear scheme: the residual with b_h
    assembled from the element convection terms (pinned separately against Eq. 9's
    pair form) is at rounding level, and the last increments fall quadratically.
    (At nu = 0.01 Newton from rest does not converge on this source.)"""
    coords, elems, fbar, _ = problem(2, 12)
    U, P, hist = steady.newton(coords, elems, 0.02, fbar, tol=1e-12)
    mom, div = steady.navier_stokes_residual(coords, elems, 0.02, fbar, U, P)
    assert mom <= 1e-10 and div <= 1e-12
    assert hist[-1] <= 1e-12 and len(hist) <= 10
    k = next(i for i, h in enumerate(hist) if h < 1e-2)
    assert hist[k + 1] <= 10 * hist[k] ** 2, hist


def test_the_stokes_solution_is_not_a_navier_stokes_solution():
    """The residual pin sees the convection term: the Stokes solution leaves it large."""
    coords, elems, fbar, _ = problem(2, 12)
    ref = pipeline.direct(coords, elems, 0.02, 0.0, fbar)
    mom, _ = steady.navier_stokes_residual(coords, elems, 0.02, fbar, ref["U"].ravel(), ref["P"])
    assert mom > 1e-3


def test_inexact_inner_solves_reach_the_steady_solution():
    """With the divergence block carried by the preconditioner, inner PCG solves to a
    relative residual of 1e-4 still reach the steady solution (flexible GMRES)."""
    from oracle import krylov
    coords, elems, fbar, w = problem(2, 12, "newton")
    ref = pipeline.direct(coords, elems, 0.01, 0.0, fbar, "newton", w)
    inner = lambda G, S: krylov.pcg(G, S, krylov.jacobi(G), rtol=1e-4)[0]   # noqa: E731
    U, P, st = steady.solve_steady(coords, elems, 0.01, fbar, "newton", w, mu_pre=1.0, pre_conv="none",
                                   restart=60, rtol=1e-11, inner=inner)
    assert st["relres"] <= 1e-11 and rel(U, ref["U"].ravel()) <= 1e-9
