"""The coupled system solved without hybridisation (cr_coupled_create,
cr_solve_coupled: preconditioned MINRES in FP64) against the CPU FP64 oracle.

* U and P reach the oracle's direct solve of Eq. 10 (1e-9 relative L2 after
  MINRES to a relative residual of 1e-12; P normalised to zero mean), in 2D
  (transient and steady Stokes) and 3D.
* One MINRES cycle takes the oracle MINRES's steps for the same target (the
  same algorithm and preconditioner; FP64 rounding moves the count by a few).
* The hybrid method's PCG needs far fewer iterations than MINRES on the same
  problem: the paper's comparison.
"""

import numpy as np
import pytest

import synth
from oracle import coupled, pipeline, topology
from paper_2101_03777_gb300 import crhyb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def case(dim, n, mu, nu=1.0):
    if dim == 2:
        coords, elems = synth.mesh2d_square(n, perturb=0.2, seed=3)
    else:
        coords, elems = synth.mesh3d_kuhn(n)
    modes = synth.fourier_modes(dim, 1)
    fbar = synth.element_means(lambda x: synth.fourier_force(x, modes), coords, elems, order=3)[None]
    mesh = crhyb.cr_mesh_load(coords, elems, need_mis=(mu == 0.0))
    system = crhyb.cr_assemble_coupled(mesh, nu, mu, torch.from_numpy(fbar).cuda())
    return coords, elems, fbar, mesh, system


def solve(system, mesh, **opts):
    cpl = crhyb.cr_coupled_create(system)
    U = torch.zeros(mesh.nf * mesh.dim, dtype=torch.float64, device="cuda")
    P = torch.zeros(mesh.ne, dtype=torch.float64, device="cuda")
    st = crhyb.cr_solve_coupled(cpl, U, P, **opts)
    return st, U.cpu().numpy(), P.cpu().numpy()


@pytest.mark.parametrize("dim,n,mu", [(2, 13, 1000.0), (2, 13, 0.0), (3, 3, 100.0)])
def test_minres_matches_the_direct_solve(dim, n, mu):
    coords, elems, fbar, mesh, system = case(dim, n, mu)
    st, U, P = solve(system, mesh, tol=1e-12, prec="fp64")
    assert st["status"] == 0 and st["relres"] <= 1e-12 and st["iterations"] > 10
    ref = pipeline.direct(coords, elems, 1.0, mu, fbar[0], dense=True)
    assert P[0] == 0.0
    assert rel(U, ref["U"].ravel()) <= 1e-9
    vol = ref["geom"]["vol"]
    assert rel(coupled.normalise_pressure(P, vol), coupled.normalise_pressure(ref["P"], vol)) <= 1e-9


def test_one_cycle_takes_the_oracle_steps():
    coords, elems, fbar, mesh, system = case(2, 16, 300.0)
    tol = 1e-8
    st, U, P = solve(system, mesh, tol=tol, prec="fp64", max_outer=1, raise_on_error=False)
    ref = pipeline.direct(coords, elems, 1.0, 300.0, fbar[0], dense=True)
    # the GPU cycle stops at |eta| <= 0.1 tol gamma_1 (the first cycle starts from x = 0)
    _, _, it, _ = coupled.solve_minres(ref["A"], ref["D"], ref["R"], rtol=0.1 * tol)
    assert abs(st["iterations"] - it) <= max(3, 0.02 * it)


def test_hybrid_pcg_needs_fewer_iterations_than_minres():
    coords, elems, fbar, mesh, system = case(2, 24, 1000.0)
    st_c, U_c, _ = solve(system, mesh, tol=1e-10, prec="fp64")
    hyb = crhyb.cr_hybridise(system, keep_fp32=False)
    W = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    st_h = crhyb.cr_solve(hyb, W, tol=1e-10, prec="fp64", persistent=True)
    U = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    P = torch.zeros(mesh.ne, dtype=torch.float64, device="cuda")
    crhyb.cr_recover_up(hyb, W, U, P)
    assert rel(U.cpu().numpy(), U_c) <= 1e-8
    assert st_h["iterations"] < st_c["iterations"]


def test_coupled_errors():
    coords, elems, fbar, mesh, system = case(2, 5, 10.0)
    cpl = crhyb.cr_coupled_create(system)
    U = torch.zeros(mesh.nf * 2, dtype=torch.float64, device="cuda")
    P = torch.zeros(mesh.ne, dtype=torch.float64, device="cuda")
    for bad in (dict(prec="ff"), dict(tol=0.0), dict(rhs=1)):
        with pytest.raises(crhyb.CrError) as ei:
            crhyb.cr_solve_coupled(cpl, U, P, **{"tol": 1e-10, "prec": "fp64", **bad})
        assert ei.value.name == "CR_ERR_ARG"
    with pytest.raises(crhyb.CrError) as ei:
        crhyb.cr_solve_coupled(cpl, U.cpu().numpy(), P.cpu().numpy(), tol=1e-10, prec="fp64")
    assert ei.value.name == "CR_ERR_ARG"
    t = topology.build_faces(elems)
    w = torch.zeros(t["nf"], 2, dtype=torch.float64, device="cuda")
    ns = crhyb.cr_assemble_coupled(mesh, 1.0, 10.0, torch.from_numpy(fbar).cuda(), conv="newton", w=w)
    with pytest.raises(crhyb.CrError) as ei:
        crhyb.cr_coupled_create(ns)
    assert ei.value.name == "CR_ERR_ARG"
    # a step limit is reported
    st, _, _ = solve(system, mesh, tol=1e-13, prec="fp64", max_iter=3, raise_on_error=False)
    assert st["status_name"] == "CR_ERR_NOT_CONVERGED" and st["iterations"] == 3


def test_second_rhs_other_k0_and_previous_level():
    """Right-hand side 1 of two, K_0 = 7, and an implicit Euler previous level:
    the same U and P as the oracle's direct solve with those choices."""
    coords, elems = synth.mesh2d_square(9, perturb=0.2, seed=8)
    fbar = np.stack([synth.element_means(lambda x, md=synth.fourier_modes(2, s): synth.fourier_force(x, md),
                                         coords, elems, order=3) for s in (2, 5)])
    mesh = crhyb.cr_mesh_load(coords, elems, k0=7)
    system = crhyb.cr_assemble_coupled(mesh, 0.5, 80.0, torch.from_numpy(fbar).cuda())
    t = topology.build_faces(elems)
    u_prev = np.random.default_rng(4).standard_normal((2, t["nf"], 2))
    crhyb.cr_system_set_previous(system, u_prev)
    cpl = crhyb.cr_coupled_create(system)
    U = torch.zeros(mesh.nf * 2, dtype=torch.float64, device="cuda")
    P = torch.zeros(mesh.ne, dtype=torch.float64, device="cuda")
    st = crhyb.cr_solve_coupled(cpl, U, P, rhs=1, tol=1e-12, prec="fp64")
    assert st["status"] == 0
    ref = pipeline.direct(coords, elems, 0.5, 80.0, fbar[1], dense=True, k0=7, u_prev=u_prev[1])
    Pn = P.cpu().numpy()
    assert Pn[7] == 0.0
    assert rel(U.cpu().numpy(), ref["U"].ravel()) <= 1e-9
    assert rel(Pn, ref["P"]) <= 1e-9
