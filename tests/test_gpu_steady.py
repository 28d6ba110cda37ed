"""Steady problems (mu = 0) through cr_solve_steady, against the oracle's direct solve.

The steady coupled system (Eq. 10 with mu = 0) is solved on the GPU by
flexible GMRES on the coupled operator, preconditioned by transient Stokes
steps of the hybrid method (SPD G, persistent PCG).  Its U and P (P
normalised to zero mean, Section 2 item 5) must match the oracle's direct
solve of the steady coupled system within 1e-9 relative L2 after a solve to a
coupled relative residual of 1e-11: steady Stokes (2D perturbed, 3D Kuhn),
steady Newton and Oseen steps (2D, nu = 0.01 and 0.05, linearised about the
seeded stream-function field), at small sizes and at 128 x 128 and 256 x 256
squares.  The number of outer steps must not grow with the mesh (the
preconditioned operator's eigenvalues are lambda/(lambda + mu)).  The oracle's
direct solves of the two larger meshes run in spawned worker processes while
the GPU solves run.
"""

import multiprocessing
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

import synth
from oracle import coupled, pipeline, topology
from paper_2101_03777_gb300 import crhyb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def problem(dim, n, conv="none"):
    if dim == 2:
        coords, elems = synth.mesh2d_square(n, 0.2, 5)
    else:
        coords, elems = synth.mesh3d_kuhn(n)
    modes = synth.fourier_modes(dim, 1)
    fbar = synth.element_means(lambda x: synth.fourier_force(x, modes), coords, elems, order=3)
    w = None
    if conv != "none":
        t = topology.build_faces(elems)
        w = synth.stream_velocity(coords[t["face_vertices"]].mean(axis=1), seed=3)
    return coords, elems, np.ascontiguousarray(fbar[None]), w


def truth(dim, n, nu, conv):
    """U and normalised P of the steady coupled system by the oracle's direct solve."""
    coords, elems, fbar, w = problem(dim, n, conv)
    ref = pipeline.direct(coords, elems, nu, 0.0, fbar[0], conv, w)
    return ref["U"].ravel(), coupled.normalise_pressure(ref["P"], ref["geom"]["vol"])


def normalise(P, coords, elems):
    """P - (1/|Omega|) sum_K |K| P_K with |K| = |det J_K| / d!."""
    X = coords[elems]
    J = X[:, 1:, :] - X[:, :1, :]
    vol = np.abs(np.linalg.det(J)) / float(np.prod(np.arange(1, J.shape[1] + 1)))
    return P - np.dot(vol, P) / vol.sum()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_steady(dim, n, nu, conv, mu_pre, prec="ff", tol=1e-11, **opts):
    coords, elems, fbar, w = problem(dim, n, conv)
    mesh = crhyb.cr_mesh_load(coords, elems)
    fb = torch.from_numpy(fbar).cuda()
    wt = torch.from_numpy(np.ascontiguousarray(w)).cuda() if w is not None else None
    sysm = crhyb.cr_assemble_coupled(mesh, nu, 0.0, fb, conv=conv, w=wt)
    pre = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, nu, mu_pre, fb), keep_fp32=False,
                             keep_ff=(prec == "ff"), keep_ff_bf16=(prec == "ff_bf16"))
    U = torch.zeros(mesh.nf * dim, dtype=torch.float64, device="cuda")
    P = torch.zeros(mesh.ne, dtype=torch.float64, device="cuda")
    st = crhyb.cr_solve_steady(sysm, pre, U, P, tol=tol, prec=prec, restart=60, **opts)
    Pn = normalise(P.cpu().numpy(), coords, elems)
    return st, U.cpu().numpy(), Pn, P.cpu().numpy()


@pytest.fixture(scope="module")
def big_truths():
    ex = ProcessPoolExecutor(max_workers=3, mp_context=multiprocessing.get_context("spawn"))
    fut = {("none", 128): ex.submit(truth, 2, 128, 1.0, "none"),
           ("none", 256): ex.submit(truth, 2, 256, 1.0, "none"),
           ("newton", 128): ex.submit(truth, 2, 128, 0.01, "newton"),
           ("newton", 256): ex.submit(truth, 2, 256, 0.01, "newton")}
    yield fut
    ex.shutdown(wait=True, cancel_futures=True)


SMALL = [(2, 24, 1.0, "none", 30.0, "ff"), (2, 24, 1.0, "none", 30.0, "fp64"), (3, 4, 1.0, "none", 30.0, "ff"),
         (2, 20, 0.01, "newton", 1.0, "ff"), (2, 16, 0.05, "oseen", 3.0, "fp64")]


@pytest.mark.parametrize("dim,n,nu,conv,mu_pre,prec", SMALL, ids=[f"{c[0]}d-{c[1]}-{c[3]}-{c[5]}" for c in SMALL])
def test_steady_matches_direct_solve(dim, n, nu, conv, mu_pre, prec):
    st, U, Pn, P = gpu_steady(dim, n, nu, conv, mu_pre, prec)
    assert st["status"] == 0 and st["relres"] <= 1e-11
    assert P[0] == 0.0                      # P_{K_0} = 0
    Uo, Po = truth(dim, n, nu, conv)
    assert rel(U, Uo) <= 1e-9 and rel(Pn, Po) <= 1e-9, (rel(U, Uo), rel(Pn, Po))


@pytest.mark.parametrize("conv,nu,mu_pre", [("none", 1.0, 30.0), ("newton", 0.01, 1.0)])
@pytest.mark.parametrize("n", [128, 256])
def test_steady_at_128_and_256_matches_direct_solve(big_truths, conv, nu, mu_pre, n):
    st, U, Pn, _ = gpu_steady(2, n, nu, conv, mu_pre)
    assert st["status"] == 0 and st["relres"] <= 1e-11
    Uo, Po = big_truths[(conv, n)].result()
    assert rel(U, Uo) <= 1e-9 and rel(Pn, Po) <= 1e-9, (rel(U, Uo), rel(Pn, Po))


def test_outer_steps_do_not_grow_with_the_mesh():
    """With accurate inner solves (1e-8) the outer count is that of the preconditioned
    operator, whose eigenvalues lambda/(lambda + mu) do not depend on the mesh (oracle:
    9 steps at 32, 64 and 128).  The default inner tolerance 1e-4 trades outer steps for
    inner work (oracle and GPU: 10, 11, 23-24 steps, 40% fewer inner iterations at 128)."""
    steps = [gpu_steady(2, n, 1.0, "none", 30.0, tol=1e-10, inner_tol=1e-8)[0]["outer"] for n in (32, 64, 128)]
    assert max(steps) - min(steps) <= 2 and max(steps) <= 12, steps


def test_steady_argument_errors():
    coords, elems, fbar, _ = problem(2, 6)
    mesh = crhyb.cr_mesh_load(coords, elems)
    fb = torch.from_numpy(fbar).cuda()
    steady = crhyb.cr_assemble_coupled(mesh, 1.0, 0.0, fb)
    transient = crhyb.cr_assemble_coupled(mesh, 1.0, 30.0, fb)
    pre = crhyb.cr_hybridise(transient, keep_ff=True)
    U = torch.zeros(mesh.nf * 2, dtype=torch.float64, device="cuda")
    P = torch.zeros(mesh.ne, dtype=torch.float64, device="cuda")
    for call in (lambda: crhyb.cr_solve_steady(transient, pre, U, P),            # not steady
                 lambda: crhyb.cr_solve_steady(steady, pre, U, P, method="pcg"),  # outer method
                 lambda: crhyb.cr_solve_steady(steady, pre, U, P, restart=1000),
                 lambda: crhyb.cr_solve_steady(steady, pre, U.cpu(), P.cpu())):  # host outputs
        with pytest.raises(crhyb.CrError) as ei:
            call()
        assert ei.value.name == "CR_ERR_ARG"
    # a steady system cannot be hybridised with E_K on a mesh loaded without M_1
    with pytest.raises(crhyb.CrError) as ei:
        crhyb.cr_hybridise(steady)
    assert ei.value.name == "CR_ERR_ARG"
    # the step limit
    st = crhyb.cr_solve_steady(steady, pre, U, P, tol=1e-14, max_iter=2, raise_on_error=False)
    assert st["status_name"] == "CR_ERR_NOT_CONVERGED" and st["outer"] == 2


def newton_truth(n, nu):
    from oracle import steady as osteady
    coords, elems, fbar, _ = problem(2, n)
    U, P, hist = osteady.newton(coords, elems, nu, fbar[0], tol=1e-12)
    return U, normalise(P, coords, elems), hist


@pytest.mark.parametrize("n", [32, 128])
def test_newton_loop_reaches_the_navier_stokes_solution(n):
    """cr_solve_newton (nu = 0.02, from rest) against the oracle's Newton loop with
    direct linear solves: the same number of steps (within one) to the increment
    tolerance, and the same end point within 1e-9."""
    nu = 0.02
    coords, elems, fbar, _ = problem(2, n)
    mesh = crhyb.cr_mesh_load(coords, elems)
    fb = torch.from_numpy(fbar[0].copy()).cuda()
    pre = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, nu, 2.0, fb[None].contiguous()), keep_fp32=False,
                             keep_ff=True)
    U = torch.zeros(mesh.nf * 2, dtype=torch.float64, device="cuda")
    P = torch.zeros(mesh.ne, dtype=torch.float64, device="cuda")
    st = crhyb.cr_solve_newton(mesh, nu, fb, pre, U, P, newton_tol=1e-10, max_newton=20, tol=1e-12, restart=60)
    assert st["status"] == 0 and st["increment"] <= 1e-10 and st["residual"] <= 1e-10, st
    Uo, Po, hist = newton_truth(n, nu)
    it_oracle = next(i + 1 for i, h in enumerate(hist) if h <= 1e-10)
    assert abs(st["iterations"] - it_oracle) <= 1, (st["iterations"], hist)
    assert rel(U.cpu().numpy(), Uo) <= 1e-9
    assert rel(normalise(P.cpu().numpy(), coords, elems), Po) <= 1e-9


def test_newton_loop_to_the_paper_tolerance():
    """The lid-driven cavity runs of the paper stop Newton at 5e-7; here on 128 x 128
    squares (nu = 0.02, homogeneous data): a handful of steps, the nonlinear residual
    of the returned iterate near the linear tolerance."""
    nu = 0.02
    coords, elems, fbar, _ = problem(2, 128)
    mesh = crhyb.cr_mesh_load(coords, elems)
    fb = torch.from_numpy(fbar[0].copy()).cuda()
    pre = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, nu, 2.0, fb[None].contiguous()), keep_fp32=False,
                             keep_ff=True)
    U = torch.zeros(mesh.nf * 2, dtype=torch.float64, device="cuda")
    P = torch.zeros(mesh.ne, dtype=torch.float64, device="cuda")
    st = crhyb.cr_solve_newton(mesh, nu, fb, pre, U, P, newton_tol=5e-7, max_newton=20, tol=1e-10, restart=60)
    assert st["status"] == 0 and st["increment"] <= 5e-7 and st["iterations"] <= 8, st
    assert st["residual"] <= 1e-8 and st["first_residual"] == pytest.approx(1.0), st


def test_deflated_inner_solves_reach_the_same_steady_solution():
    """Ritz vectors of the preconditioning system's G (which every inner solve shares)
    deflate the inner float-float Chebyshev PCG: the steady solution at 128 x 128 is the
    undeflated one within 1e-9, with fewer inner iterations."""
    coords, elems, fbar, w = problem(2, 128, "newton")
    mesh = crhyb.cr_mesh_load(coords, elems)
    fb = torch.from_numpy(fbar).cuda()
    wt = torch.from_numpy(np.ascontiguousarray(w)).cuda()
    sysm = crhyb.cr_assemble_coupled(mesh, 0.01, 0.0, fb, conv="newton", w=wt)
    pre = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, 0.01, 1.0, fb), keep_fp32=True, keep_bf16=True,
                             keep_ff=True)
    cheb = dict(precond="chebyshev", poly_degree=8, poly_ratio=1000.0)
    d, _ = crhyb.cr_deflation_lanczos(pre, 120, 8, **cheb)
    out = []
    for defl in (None, d):
        U = torch.zeros(mesh.nf * 2, dtype=torch.float64, device="cuda")
        P = torch.zeros(mesh.ne, dtype=torch.float64, device="cuda")
        st = crhyb.cr_solve_steady(sysm, pre, U, P, tol=1e-11, prec="ff", poly_prec="bf16", restart=60,
                                   deflation=defl, **cheb)
        assert st["status"] == 0 and st["relres"] <= 1e-11
        out.append((st, U.cpu().numpy()))
    (st0, U0), (st1, U1) = out
    assert rel(U1, U0) <= 1e-9
    assert st1["iterations"] < st0["iterations"], (st1["iterations"], st0["iterations"])
    # a space of another G is refused
    other = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, 0.01, 2.0, fb), keep_ff=True)
    d2, _ = crhyb.cr_deflation_lanczos(other, 20, 2)
    with pytest.raises(crhyb.CrError) as ei:
        crhyb.cr_solve_steady(sysm, pre, U, P, prec="ff", deflation=d2, **cheb)
    assert ei.value.name == "CR_ERR_ARG"
