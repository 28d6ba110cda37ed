"""Batched solves (many meshes of uneven size x several right-hand sides in one
persistent launch) against the CPU FP64 oracle and against the one-problem
solve, through the C-ABI.

Tolerances as in test_gpu_parity: U and P (P normalised to zero mean) within
1e-9 relative L2 of the oracle's direct solve of the coupled system after
float-float or FP64 PCG to a relative residual of 1e-13; 1e-8 with BF16 low
parts of G.  The batch is the workload of the batched benchmark scaled down:
perturbed 2D meshes with n drawn log-uniformly (seeded), up to 4 right-hand
sides each, with tile counts from 1 to several per problem and ragged tails.
"""

import numpy as np
import pytest

import synth
from oracle import coupled, pipeline
from paper_2101_03777_gb300 import crhyb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def small_batch(count=6, lo=3, hi=24, nrhs=(1, 4, 2, 3, 4, 1)):
    probs = synth.batch_problems(count=count, nrhs=4, lo=lo, hi=hi, seed=2)
    for p, r in zip(probs, nrhs):
        p["fbar"] = np.ascontiguousarray(p["fbar"][:r])
    return probs


def hybridise_all(probs):
    out = []
    for p in probs:
        mesh = crhyb.cr_mesh_load(p["coords"], p["elems"])
        fb = torch.from_numpy(p["fbar"]).cuda()
        sysm = crhyb.cr_assemble_coupled(mesh, p["nu"], p["mu"], fb)
        out.append(crhyb.cr_hybridise(sysm, keep_fp32=True, keep_ff=True, keep_ff_bf16=True))
    return out


@pytest.mark.parametrize("prec,tol,grouping", [("ff", 1e-9, 1), ("fp64", 1e-9, 1), ("ff_bf16", 1e-8, 1),
                                               ("ff", 1e-9, 2), ("fp64", 1e-9, 2), ("ff", 1e-9, 3),
                                               ("fp64", 1e-9, 3)])
def test_batch_matches_oracle_per_pair(prec, tol, grouping):
    probs = small_batch()
    hybs = hybridise_all(probs)
    batch = crhyb.cr_batch_create(hybs, prec=prec, rhs_grouping=grouping)
    info = batch.info()
    npairs = sum(p["fbar"].shape[0] for p in probs)
    nsys = {1: len(probs), 2: npairs, 3: sum((p["fbar"].shape[0] + 1) // 2 for p in probs)}[grouping]
    assert info["nsys"] == nsys and info["grid"] >= 1
    Ws = [torch.zeros(h.system.nrhs * h.n, dtype=torch.float64, device="cuda") for h in hybs]
    stats = crhyb.cr_solve_batched(batch, Ws, tol=1e-13, max_iter=100000)
    j = 0
    for p, h, W in zip(probs, hybs, Ws):
        for r in range(h.system.nrhs):
            st = stats[j]
            j += 1
            assert st["status"] == 0 and st["relres"] <= 1e-13
            ref = pipeline.direct(p["coords"], p["elems"], p["nu"], p["mu"], p["fbar"][r], dense=True)
            Wr = W[r * h.n:(r + 1) * h.n].contiguous()
            U = torch.zeros(h.n, dtype=torch.float64, device="cuda")
            P = torch.zeros(h.mesh.ne, dtype=torch.float64, device="cuda")
            crhyb.cr_recover_up(h, Wr, U, P, rhs=r)
            assert rel(U.cpu().numpy(), ref["U"].ravel()) <= tol
            assert rel(P.cpu().numpy(), coupled.normalise_pressure(ref["P"], ref["geom"]["vol"])) <= tol


def test_batch_matches_single_solves_and_autotunes():
    """Each pair of the batch takes the iterations of its own one-problem solve
    (to rounding of the dot products) and converges to the same W."""
    probs = small_batch()
    hybs = hybridise_all(probs)
    batch = crhyb.cr_batch_create(hybs, prec="ff", autotune=True)
    Ws = [torch.zeros(h.system.nrhs * h.n, dtype=torch.float64, device="cuda") for h in hybs]
    stats = crhyb.cr_solve_batched(batch, Ws, tol=1e-11)
    info = batch.info()
    assert 1 <= info["blocks_per_sm"] <= 7
    # any of the three groupings may win
    assert info["nsys"] in (len(probs), sum(h.system.nrhs for h in hybs), sum((h.system.nrhs + 1) // 2 for h in hybs))
    stats2 = crhyb.cr_solve_batched(batch, Ws, tol=1e-11)      # a second solve reuses the tuned plan
    assert [s["iterations"] for s in stats2] == [s["iterations"] for s in stats]
    j = 0
    for h, W in zip(hybs, Ws):
        for r in range(h.system.nrhs):
            W1 = torch.zeros(h.n, dtype=torch.float64, device="cuda")
            st1 = crhyb.cr_solve(h, W1, rhs=r, tol=1e-11, prec="ff", persistent=True)
            assert abs(st1["iterations"] - stats[j]["iterations"]) <= 0.02 * st1["iterations"] + 2
            assert rel(W[r * h.n:(r + 1) * h.n].cpu().numpy(), W1.cpu().numpy()) <= 1e-9
            j += 1


def test_batch_warm_start_limits_and_errors():
    probs = small_batch(count=3, nrhs=(2, 1, 3))
    hybs = hybridise_all(probs)
    batch = crhyb.cr_batch_create(hybs, prec="fp64")
    Ws = [torch.zeros(h.system.nrhs * h.n, dtype=torch.float64, device="cuda") for h in hybs]
    st = crhyb.cr_solve_batched(batch, Ws, tol=1e-13, max_iter=5, raise_on_error=False)
    assert all(s["status"] == -4 and s["iterations"] == 5 for s in st)
    crhyb.cr_solve_batched(batch, Ws, tol=1e-12)
    st = crhyb.cr_solve_batched(batch, Ws, tol=1e-10, use_x0=True)
    assert all(s["status"] == 0 and s["iterations"] <= 1 for s in st)
    # mu = 0 has no SPD G: refused
    coords, elems = synth.mesh2d_square(3, 0.2, 2)
    mesh = crhyb.cr_mesh_load(coords, elems, need_mis=True)
    h0 = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, 1.0, 0.0, np.ones((1, elems.shape[0], 2))))
    with pytest.raises(crhyb.CrError) as ei:
        crhyb.cr_batch_create([h0], prec="fp64")
    assert ei.value.name == "CR_ERR_ARG"
    with pytest.raises(crhyb.CrError):
        crhyb.cr_batch_create(hybs, prec="mixed")
