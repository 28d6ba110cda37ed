"""A Navier-Stokes implicit Euler step solved by Newton's method, composed from
the library's calls (Section 3.1 Newton linearisation; Section 4.3 Newton
loop): each Newton iterate assembles the linearisation about the current
velocity (cr_assemble_coupled with conv = NEWTON), carries the previous time
level (cr_system_set_previous), hybridises, solves with the Stokes-
preconditioned flexible GMRES and recovers the next iterate.

Checked against the oracle's Newton iterates (its direct solve of the same
linear systems) to 1e-9, and for the quadratic convergence Newton's method
has: each correction is at most a fixed multiple of the square of the last.
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


def test_newton_iterates_of_a_navier_stokes_time_step():
    n, nu, mu = 14, 0.01, 100.0                # Re = 100, dt = 1e-2
    coords, elems = synth.mesh2d_square(n, perturb=0.1, seed=6)
    t = topology.build_faces(elems)
    nf = t["nf"]
    modes = synth.fourier_modes(2, 1)
    fbar = 20.0 * synth.element_means(lambda x: synth.fourier_force(x, modes), coords, elems, order=3)[None]
    u_n = synth.stream_velocity(coords[t["face_vertices"]].mean(axis=1), seed=3)[None]   # previous level
    mesh = crhyb.cr_mesh_load(coords, elems)
    fb = torch.from_numpy(fbar).cuda()
    pre = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, nu, mu, fb), keep_fp32=False, keep_ff=True)
    w_gpu = torch.from_numpy(u_n[0].copy()).cuda()    # Newton starts from the previous level
    w_ref = u_n[0].copy()
    corrections = []
    for k in range(5):
        system = crhyb.cr_assemble_coupled(mesh, nu, mu, fb, conv="newton", w=w_gpu)
        crhyb.cr_system_set_previous(system, u_n)
        hyb = crhyb.cr_hybridise(system, keep_fp32=False)
        W = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
        st = crhyb.cr_solve_preconditioned(hyb, pre, W, tol=1e-13, prec="ff")
        assert st["status"] == 0
        U = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
        P = torch.zeros(mesh.ne, dtype=torch.float64, device="cuda")
        crhyb.cr_recover_up(hyb, W, U, P, normalise_p=True)
        ref = pipeline.direct(coords, elems, nu, mu, fbar[0], "newton", w_ref, dense=True, u_prev=u_n[0])
        Un = U.cpu().numpy()
        assert rel(Un, ref["U"].ravel()) <= 1e-9
        assert rel(P.cpu().numpy(), coupled.normalise_pressure(ref["P"], ref["geom"]["vol"])) <= 1e-9
        corrections.append(np.linalg.norm(Un - w_gpu.cpu().numpy().ravel()) / np.linalg.norm(Un))
        w_gpu = U.reshape(nf, 2).contiguous()
        w_ref = ref["U"].reshape(nf, 2)
    # quadratic convergence while the Newton error is above the linear solves' rounding:
    # e_{k+1} <= e_k^2 (the oracle's ratios e_{k+1}/e_k^2 are about 0.08 here)
    e = corrections
    for k in range(3):
        assert e[k + 1] <= e[k] ** 2, e
    assert e[3] < 1e-7 and e[4] < 1e-10, e
