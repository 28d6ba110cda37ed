"""Implicit Euler time steps (mu = 1/dt) on the GPU against the CPU FP64
oracle, through the C-ABI: cr_system_set_previous makes the right-hand side of
the next cr_hybridise / cr_recover_up carry the lumped mass of the previous
time level (Section 2 with the mass of Section 3.1).

Tolerances as in test_gpu_parity: 1e-9 relative L2 in U and P (P normalised
to zero mean) after PCG to 1e-13; the steps of a loop accumulate no more than
rounding, so ten steps stay within 1e-9 too.
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


def setup(dim, n, nrhs=1, mu=200.0, nu=1.0):
    if dim == 2:
        coords, elems = synth.mesh2d_square(n, perturb=0.2, seed=4)
    else:
        coords, elems = synth.mesh3d_kuhn(n)
    fbar = np.stack([synth.element_means(lambda x, md=synth.fourier_modes(dim, 1 + 1000 * j): synth.fourier_force(x, md),
                                         coords, elems, order=3) for j in range(nrhs)])
    mesh = crhyb.cr_mesh_load(coords, elems)
    system = crhyb.cr_assemble_coupled(mesh, nu, mu, torch.from_numpy(fbar).cuda())
    return coords, elems, fbar, mesh, system, mu, nu


def step(system, u_prev, prec="ff", rhs_count=1):
    """One implicit Euler step of every right-hand side: (U [nrhs, n], P [nrhs, ne], stats)."""
    crhyb.cr_system_set_previous(system, u_prev)
    hyb = crhyb.cr_hybridise(system, keep_fp32=False, keep_ff=True)
    n, ne = hyb.n, hyb.mesh.ne
    U = torch.zeros(rhs_count, n, dtype=torch.float64, device="cuda")
    P = torch.zeros(rhs_count, ne, dtype=torch.float64, device="cuda")
    stats = []
    for r in range(rhs_count):
        W = torch.zeros(n, dtype=torch.float64, device="cuda")
        stats.append(crhyb.cr_solve(hyb, W, rhs=r, tol=1e-13, prec=prec, persistent=True))
        crhyb.cr_recover_up(hyb, W, U[r], P[r], rhs=r, normalise_p=True)
    return U, P, stats


@pytest.mark.parametrize("dim,n,prec", [(2, 11, "ff"), (2, 11, "fp64"), (3, 3, "fp64")])
def test_one_step_matches_oracle(dim, n, prec):
    coords, elems, fbar, mesh, system, mu, nu = setup(dim, n)
    t = topology.build_faces(elems)
    u_prev = np.random.default_rng(5).standard_normal((1, t["nf"], dim))
    U, P, st = step(system, torch.from_numpy(u_prev).cuda(), prec)
    assert st[0]["status"] == 0
    ref = pipeline.direct(coords, elems, nu, mu, fbar[0], dense=True, u_prev=u_prev[0])
    assert rel(U[0].cpu().numpy(), ref["U"].ravel()) <= 1e-9
    assert rel(P[0].cpu().numpy(), coupled.normalise_pressure(ref["P"], ref["geom"]["vol"])) <= 1e-9


def test_steady_solution_is_a_fixed_point_on_the_gpu():
    coords, elems, fbar, mesh, system, mu, nu = setup(2, 9)
    steady = pipeline.direct(coords, elems, nu, 0.0, fbar[0], dense=True)
    U, P, _ = step(system, steady["U"].reshape(1, -1, 2).copy())      # host pointer path
    assert rel(U[0].cpu().numpy(), steady["U"].ravel()) <= 1e-9
    assert rel(P[0].cpu().numpy(), coupled.normalise_pressure(steady["P"], steady["geom"]["vol"])) <= 1e-9


def test_ten_steps_with_two_right_hand_sides_follow_the_oracle():
    coords, elems, fbar, mesh, system, mu, nu = setup(2, 8, nrhs=2, mu=50.0)
    nf = mesh.nf
    u_dev = torch.zeros(2, nf, 2, dtype=torch.float64, device="cuda")
    u_ref = [np.zeros((nf, 2)), np.zeros((nf, 2))]
    for k in range(10):
        U, P, st = step(system, u_dev, "ff", rhs_count=2)
        assert all(s["status"] == 0 for s in st)
        u_dev = U.reshape(2, nf, 2).contiguous()
        for r in range(2):
            out = pipeline.direct(coords, elems, nu, mu, fbar[r], dense=True, u_prev=u_ref[r])
            u_ref[r] = out["U"].reshape(-1, 2)
            if k == 9:
                assert rel(U[r].cpu().numpy(), u_ref[r].ravel()) <= 1e-9
                assert rel(P[r].cpu().numpy(), coupled.normalise_pressure(out["P"], out["geom"]["vol"])) <= 1e-9
    # the loop approaches the steady state from zero: u^10 lies between 0 and it
    steady = pipeline.direct(coords, elems, nu, 0.0, fbar[0], dense=True)["U"].ravel()
    d10 = np.linalg.norm(U[0].cpu().numpy() - steady)
    assert 0.0 < d10 < np.linalg.norm(steady)


def test_previous_level_off_and_errors():
    coords, elems, fbar, mesh, system, mu, nu = setup(2, 6)
    t = topology.build_faces(elems)
    u_prev = np.random.default_rng(2).standard_normal((1, t["nf"], 2))
    U1, _, _ = step(system, u_prev)
    U0, _, _ = step(system, None)                                  # turned off again
    ref0 = pipeline.direct(coords, elems, nu, mu, fbar[0], dense=True)
    assert rel(U0[0].cpu().numpy(), ref0["U"].ravel()) <= 1e-9
    assert rel(U1[0].cpu().numpy(), ref0["U"].ravel()) > 1e-3
    # mu = 0 has no time step
    steady = crhyb.cr_assemble_coupled(crhyb.cr_mesh_load(coords, elems, need_mis=True), nu, 0.0, fbar)
    with pytest.raises(crhyb.CrError) as ei:
        crhyb.cr_system_set_previous(steady, u_prev)
    assert ei.value.name == "CR_ERR_ARG"
    with pytest.raises(ValueError):
        crhyb.cr_system_set_previous(system, np.zeros(5))
