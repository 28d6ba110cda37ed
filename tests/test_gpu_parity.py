"""GPU parity: the CUDA library against the CPU FP64 oracle, through the C-ABI.

Tolerances (relative L2 unless stated):
  * G and S after hybridisation: 1e-12 of max |G|, |S| (same FP64 formulas,
    different rounding order);
  * U and P (P normalised to zero mean) after an FP64 solve to a relative
    residual of 1e-13: 1e-9; after mixed-precision refinement to 1e-13: 1e-8;
  * element blocks A_K, D_K, R_K: 1e-12 of the largest entry.
Meshes span several thread blocks and a ragged tail (element and face counts
that are not multiples of the block sizes).
"""

import numpy as np
import pytest

import synth
from oracle import coupled, pipeline, topology
from oracle import hybrid as ohyb
from paper_2101_03777_gb300 import crhyb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make_case(name):
    """(coords, elems, nu, mu, conv, fbar [nrhs, ne, d], w or None)."""
    if name == "cfg1":
        p = synth.config_problem("cfg1")
        return p["coords"], p["elems"], p["nu"], p["mu"], "none", p["fbar"], None
    if name == "2d_perturbed_37":
        p = synth.config_problem("cfg2", n=37, nrhs=2)
        return p["coords"], p["elems"], p["nu"], p["mu"], "none", p["fbar"], None
    if name == "3d_kuhn_5":
        p = synth.config_problem("cfg3", n=5)
        return p["coords"], p["elems"], p["nu"], p["mu"], "none", p["fbar"], None
    if name in ("ns_newton_9", "ns_oseen_9"):
        coords, elems = synth.mesh2d_square(9, 0.1, 4)
        t = topology.build_faces(elems)
        w = synth.stream_velocity(coords[t["face_vertices"]].mean(axis=1), seed=3)
        modes = synth.fourier_modes(2, 1)
        fbar = synth.element_means(lambda x: synth.fourier_force(x, modes), coords, elems, order=3)[None]
        return coords, elems, 0.01, 100.0, name.split("_")[1], fbar, w
    if name == "steady_stokes_3":
        coords, elems = synth.mesh2d_square(3, 0.2, 2)
        modes = synth.fourier_modes(2, 1)
        fbar = synth.element_means(lambda x: synth.fourier_force(x, modes), coords, elems, order=3)[None]
        return coords, elems, 1.0, 0.0, "none", fbar, None
    if name == "steady_newton_3":
        coords, elems = synth.mesh2d_square(3, 0.2, 2)
        t = topology.build_faces(elems)
        w = synth.stream_velocity(coords[t["face_vertices"]].mean(axis=1), seed=3)
        modes = synth.fourier_modes(2, 1)
        fbar = synth.element_means(lambda x: synth.fourier_force(x, modes), coords, elems, order=3)[None]
        return coords, elems, 0.05, 0.0, "newton", fbar, w
    raise ValueError(name)


def gpu_setup(case, keep_bf16=False, k0=0, keep_ff=True, keep_ff_bf16=True):
    coords, elems, nu, mu, conv, fbar, w = case
    mesh = crhyb.cr_mesh_load(coords, elems, k0=k0, need_mis=(mu == 0.0))
    fb = torch.from_numpy(np.ascontiguousarray(fbar)).cuda()
    wt = torch.from_numpy(np.ascontiguousarray(w)).cuda() if w is not None else None
    system = crhyb.cr_assemble_coupled(mesh, nu, mu, fb, conv=conv, w=wt)
    hyb = crhyb.cr_hybridise(system, keep_fp32=True, keep_bf16=keep_bf16, keep_ff=keep_ff,
                             keep_ff_bf16=keep_ff_bf16)
    return mesh, system, hyb


def oracle_hybrid(case, rhs=0, k0=0):
    coords, elems, nu, mu, conv, fbar, w = case
    return pipeline.hybrid(coords, elems, nu, mu, fbar[rhs], conv, w, k0=k0, method="direct")


CASES = ["cfg1", "2d_perturbed_37", "3d_kuhn_5", "ns_newton_9", "ns_oseen_9", "steady_stokes_3", "steady_newton_3"]


@pytest.mark.parametrize("name", CASES)
def test_topology_matches_oracle(name):
    case = make_case(name)
    mesh, _, _ = gpu_setup(case)
    t = topology.build_faces(case[1])
    assert mesh.nf == t["nf"] and mesh.nf_ext == t["n_exterior"]
    assert np.array_equal(crhyb.cr_mesh_faces(mesh), t["face_vertices"])
    fe, fl = crhyb.cr_mesh_face_elements(mesh)
    assert np.array_equal(fe, t["face_elems"]) and np.array_equal(fl, t["face_local"])
    if case[3] == 0.0:
        assert np.array_equal(crhyb.cr_mesh_mis(mesh), topology.maximal_independent_set(t))


@pytest.mark.parametrize("name", CASES)
def test_element_blocks_match_oracle(name):
    coords, elems, nu, mu, conv, fbar, w = case = make_case(name)
    mesh = crhyb.cr_mesh_load(coords, elems, need_mis=(mu == 0.0))
    d = coords.shape[1]
    L = (d + 1) * d
    nrhs = fbar.shape[0]
    out = np.zeros((elems.shape[0], L * L + L + nrhs * L))
    crhyb.cr_assemble_coupled(mesh, nu, mu, fbar, conv=conv, w=w, blocks_out=out)
    topo, geom, A_K, D_K, R_K = pipeline.setup(coords, elems, nu, mu, fbar[0], conv, w)
    A = out[:, :L * L].reshape(-1, L, L)
    assert np.abs(A - A_K).max() <= 1e-12 * np.abs(A_K).max()
    assert np.abs(out[:, L * L:L * L + L] - D_K).max() <= 1e-12 * np.abs(D_K).max()
    for r in range(nrhs):
        _, _, _, _, Rr = pipeline.setup(coords, elems, nu, mu, fbar[r], conv, w)
        got = out[:, L * L + L + r * L:L * L + L + (r + 1) * L]
        assert np.abs(got - Rr).max() <= 1e-12 * np.abs(Rr).max()


@pytest.mark.parametrize("name", CASES)
def test_hybridised_system_matches_oracle(name):
    case = make_case(name)
    _, system, hyb = gpu_setup(case)
    cols, vals, S = crhyb.cr_hybrid_export(hyb)
    G = crhyb.ell_to_csr(cols, vals)
    for r in range(system.nrhs):
        o = oracle_hybrid(case, rhs=r)
        Go = o["hyb"]["G"]
        if r == 0:
            assert abs(G - Go).max() <= 1e-12 * abs(Go).max()
            # every ELL padding slot is zero and points at its own row
            pad = cols[1:] == np.arange(cols.shape[1])[None, :]
            assert np.all(vals[1:][np.broadcast_to(pad[:, None, None, :], vals[1:].shape)] == 0.0)
        So = o["hyb"]["S"].reshape(-1, case[0].shape[1])
        assert np.abs(S[r] - So).max() <= 1e-12 * np.abs(So).max()


def solve_and_recover(hyb, rhs, **opts):
    n, ne = hyb.n, hyb.mesh.ne
    W = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = crhyb.cr_solve(hyb, W, rhs=rhs, **opts)
    U = torch.zeros(n, dtype=torch.float64, device="cuda")
    P = torch.zeros(ne, dtype=torch.float64, device="cuda")
    jump = crhyb.cr_recover_up(hyb, W, U, P, rhs=rhs, normalise_p=True, jump=True)
    return st, W.cpu().numpy(), U.cpu().numpy(), P.cpu().numpy(), jump


SOLVE_CASES = [
    ("cfg1", dict(method="pcg", prec="fp64"), 1e-9),
    ("cfg1", dict(method="pcg", prec="mixed"), 1e-8),
    ("cfg1", dict(method="pcg", prec="fp64", use_graph=True), 1e-9),
    ("2d_perturbed_37", dict(method="pcg", prec="fp64"), 1e-9),
    ("2d_perturbed_37", dict(method="pcg", prec="mixed", use_graph=True), 1e-8),
    ("2d_perturbed_37", dict(method="gmres", prec="fp64"), 1e-9),
    ("3d_kuhn_5", dict(method="pcg", prec="fp64"), 1e-9),
    ("3d_kuhn_5", dict(method="pcg", prec="mixed"), 1e-8),
    # float-float PCG with FP64 reliable updates (FP64-class accuracy)
    ("cfg1", dict(method="pcg", prec="ff"), 1e-9),
    ("2d_perturbed_37", dict(method="pcg", prec="ff"), 1e-9),
    ("2d_perturbed_37", dict(method="pcg", prec="ff", use_graph=True), 1e-9),
    ("2d_perturbed_37", dict(method="pcg", prec="ff_bf16"), 1e-8),
    ("3d_kuhn_5", dict(method="pcg", prec="ff"), 1e-9),
    ("3d_kuhn_5", dict(method="pcg", prec="ff_bf16", use_graph=True), 1e-8),
    # the same iterations in one cooperative persistent launch
    ("cfg1", dict(method="pcg", prec="fp64", persistent=True), 1e-9),
    ("cfg1", dict(method="pcg", prec="ff", persistent=True), 1e-9),
    ("2d_perturbed_37", dict(method="pcg", prec="fp64", persistent=True), 1e-9),
    ("2d_perturbed_37", dict(method="pcg", prec="ff", persistent=True), 1e-9),
    ("2d_perturbed_37", dict(method="pcg", prec="ff_bf16", persistent=True), 1e-8),
    ("3d_kuhn_5", dict(method="pcg", prec="fp64", persistent=True), 1e-9),
    ("3d_kuhn_5", dict(method="pcg", prec="ff", persistent=True), 1e-9),
    ("ns_newton_9", dict(method="gmres", prec="fp64"), 1e-9),
    # BiCGStab (nonsymmetric Newton/Oseen systems, and the SPD case)
    ("ns_newton_9", dict(method="bicgstab", prec="fp64"), 1e-9),
    ("ns_oseen_9", dict(method="bicgstab", prec="fp64"), 1e-9),
    ("2d_perturbed_37", dict(method="bicgstab", prec="fp64", use_graph=True), 1e-9),
    ("ns_newton_9", dict(method="gmres", prec="mixed"), 1e-8),
    ("ns_oseen_9", dict(method="gmres", prec="mixed"), 1e-8),
    # steady (mu = 0): full GMRES (restart >= N = 42), Jacobi-GMRES(30) stagnates there
    ("steady_stokes_3", dict(method="gmres", prec="fp64", restart=64), 1e-9),
    ("steady_newton_3", dict(method="gmres", prec="fp64", restart=64), 1e-9),
]


@pytest.mark.parametrize("name,opts,tol", SOLVE_CASES, ids=[f"{c[0]}-{c[1]['method']}-{c[1]['prec']}-{i}"
                                                            for i, c in enumerate(SOLVE_CASES)])
def test_solution_matches_coupled_direct_solve(name, opts, tol):
    case = make_case(name)
    coords, elems, nu, mu, conv, fbar, w = case
    _, system, hyb = gpu_setup(case, keep_bf16=opts.get("prec") == "mixed_bf16")
    ref = pipeline.direct(coords, elems, nu, mu, fbar[0], conv, w, dense=elems.shape[0] < 3000)
    vol = ref["geom"]["vol"]
    st, W, U, P, jump = solve_and_recover(hyb, 0, tol=1e-13, max_iter=200000, **opts)
    assert st["status"] == 0 and st["relres"] <= 2e-13
    assert rel(U, ref["U"].ravel()) <= tol
    assert rel(P, coupled.normalise_pressure(ref["P"], vol)) <= tol
    assert jump <= 1e-8 * np.abs(U).max()
    # discrete divergence-free element by element (Section 3.2, item 2)
    t, g = ref["topo"], ref["geom"]
    Ul = np.where((t["elem_face"] >= 0)[:, :, None], U.reshape(-1, coords.shape[1])[np.maximum(t["elem_face"], 0)], 0)
    div = np.einsum("kld,kld->k", Ul, g["a"])
    assert np.abs(div).max() <= 1e-9 * np.abs(g["a"]).max() * np.abs(U).max()


def stokes_preconditioner(mesh, case, keep_ff=True, keep_ff_bf16=True, keep_bf16=True):
    """The transient Stokes system with the case's nu and mu on the same mesh."""
    coords, elems, nu, mu, conv, fbar, w = case
    fb = torch.from_numpy(np.ascontiguousarray(fbar)).cuda()
    return crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, nu, mu, fb), keep_fp32=False, keep_ff=keep_ff,
                              keep_ff_bf16=keep_ff_bf16, keep_bf16=keep_bf16)


CHEB_INNER = dict(precond="chebyshev", poly_degree=8, poly_ratio=1000.0)
FGMRES_CASES = [("ns_newton_9", "ff", {}), ("ns_newton_9", "fp64", {}), ("ns_oseen_9", "ff", {}),
                ("ns_newton_9", "ff_bf16", {}),
                # inner solves by the Chebyshev-preconditioned PCG: FP64, float-float with BF16 steps
                ("ns_newton_9", "fp64", CHEB_INNER), ("ns_newton_9", "ff", dict(CHEB_INNER, poly_prec="bf16")),
                ("ns_oseen_9", "ff", dict(CHEB_INNER, poly_prec="fp32"))]


@pytest.mark.parametrize("name,prec,extra", FGMRES_CASES,
                         ids=[f"{c[0]}-{c[1]}-{c[2].get('precond', 'jacobi')}-{c[2].get('poly_prec', 'same')}"
                              for c in FGMRES_CASES])
def test_stokes_preconditioned_fgmres_matches_direct_solve(name, prec, extra):
    """Flexible GMRES preconditioned by inner PCG solves with the Stokes G (Jacobi, or
    Chebyshev in FP64 or float-float with reduced-precision steps): the outer residual
    is FP64, so every inner precision reaches the FP64 bound."""
    case = make_case(name)
    coords, elems, nu, mu, conv, fbar, w = case
    mesh, _, hyb = gpu_setup(case)
    pre = stokes_preconditioner(mesh, case)
    ref = pipeline.direct(coords, elems, nu, mu, fbar[0], conv, w, dense=True)
    W = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    st = crhyb.cr_solve_preconditioned(hyb, pre, W, tol=1e-13, prec=prec, **extra)
    assert st["status"] == 0 and st["relres"] <= 1e-12
    assert 1 <= st["outer"] <= 30 and st["iterations"] >= st["outer"]
    U = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    P = torch.zeros(mesh.ne, dtype=torch.float64, device="cuda")
    crhyb.cr_recover_up(hyb, W, U, P, normalise_p=True)
    assert rel(U.cpu().numpy(), ref["U"].ravel()) <= 1e-9
    assert rel(P.cpu().numpy(), coupled.normalise_pressure(ref["P"], ref["geom"]["vol"])) <= 1e-9
    # warm start from the solution: no step needed
    st2 = crhyb.cr_solve_preconditioned(hyb, pre, W, tol=1e-12, prec=prec, use_x0=True, **extra)
    assert st2["status"] == 0 and st2["outer"] == 0


def test_stokes_preconditioned_second_rhs():
    """Right-hand side 1 of a two-right-hand-side Newton system."""
    coords, elems = synth.mesh2d_square(9, 0.1, 4)
    t = topology.build_faces(elems)
    w = synth.stream_velocity(coords[t["face_vertices"]].mean(axis=1), seed=3)
    fbar = np.stack([synth.element_means(lambda x, md=synth.fourier_modes(2, s): synth.fourier_force(x, md),
                                         coords, elems, order=3) for s in (1, 6)])
    case = (coords, elems, 0.01, 100.0, "newton", fbar, w)
    mesh, _, hyb = gpu_setup(case)
    pre = stokes_preconditioner(mesh, case)
    W = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    st = crhyb.cr_solve_preconditioned(hyb, pre, W, rhs=1, tol=1e-13, prec="ff")
    assert st["status"] == 0
    U = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    P = torch.zeros(mesh.ne, dtype=torch.float64, device="cuda")
    crhyb.cr_recover_up(hyb, W, U, P, rhs=1, normalise_p=True)
    ref = pipeline.direct(coords, elems, 0.01, 100.0, fbar[1], "newton", w, dense=True)
    assert rel(U.cpu().numpy(), ref["U"].ravel()) <= 1e-9
    assert rel(P.cpu().numpy(), coupled.normalise_pressure(ref["P"], ref["geom"]["vol"])) <= 1e-9


def test_stokes_preconditioned_steps_do_not_grow_with_the_mesh():
    """The GMRES steps of the Stokes-preconditioned Newton solve stay bounded as
    the mesh is refined (G_pre^{-1} G differs from I by the convection term),
    while Jacobi-GMRES(30) needs ever more (and stalls beyond about 64x64)."""
    steps = []
    for n in (16, 48):
        p = synth.config_problem("cfg5", n=n)
        t = topology.build_faces(p["elems"])
        w = synth.stream_velocity(p["coords"][t["face_vertices"]].mean(axis=1), seed=3)
        case = (p["coords"], p["elems"], p["nu"], 1000.0, "newton", p["fbar"], w)
        mesh, _, hyb = gpu_setup(case)
        pre = stokes_preconditioner(mesh, case)
        W = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
        st = crhyb.cr_solve_preconditioned(hyb, pre, W, tol=1e-10, prec="ff")
        assert st["status"] == 0 and st["relres"] <= 1e-9
        # the oracle's G and S, for the residual of the returned W
        topo, geom, A_K, D_K, R_K = pipeline.setup(p["coords"], p["elems"], p["nu"], 1000.0, p["fbar"][0],
                                                   "newton", w)
        h = ohyb.hybridise(topo, A_K, D_K, R_K, 1000.0)
        Wn = W.cpu().numpy()
        assert np.linalg.norm(h["S"] - h["G"] @ Wn) <= 1e-9 * np.linalg.norm(h["S"])
        steps.append(st["outer"])
    assert max(steps) <= 20 and steps[1] <= steps[0] + 4


def test_stokes_preconditioned_error_paths():
    case = make_case("ns_newton_9")
    mesh, _, hyb = gpu_setup(case)
    W = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    # a preconditioner on another mesh handle, or one that is not SPD, is refused
    other, _, _ = gpu_setup(case)
    for bad in (stokes_preconditioner(other, case), hyb):
        with pytest.raises(crhyb.CrError) as ei:
            crhyb.cr_solve_preconditioned(hyb, bad, W, tol=1e-10)
        assert ei.value.name == "CR_ERR_ARG"
    pre = stokes_preconditioner(mesh, case, keep_ff=False, keep_ff_bf16=False)
    for opts in (dict(method="pcg"), dict(prec="mixed"), dict(restart=0, tol=0.0), dict(prec="ff")):
        with pytest.raises(crhyb.CrError) as ei:
            crhyb.cr_solve_preconditioned(hyb, pre, W, **{"tol": 1e-10, **opts})
        assert ei.value.name == "CR_ERR_ARG"
    # a step limit is reported with the last iterate's residual
    st = crhyb.cr_solve_preconditioned(hyb, pre, W, tol=1e-13, prec="fp64", max_iter=2, raise_on_error=False)
    assert st["status_name"] == "CR_ERR_NOT_CONVERGED" and st["outer"] == 2 and 0 < st["relres"] < 1


@pytest.mark.parametrize("name", ["cfg1", "3d_kuhn_5"])
def test_bf16_values_converge_or_report(name):
    """BF16 values of G are kept only where the refinement still converges: the
    solve either matches the oracle or returns a non-convergence status, never
    a wrong answer with CR_OK."""
    case = make_case(name)
    coords, elems, nu, mu, conv, fbar, w = case
    _, system, hyb = gpu_setup(case, keep_bf16=True)
    ref = pipeline.direct(coords, elems, nu, mu, fbar[0], conv, w, dense=elems.shape[0] < 3000)
    n = hyb.n
    W = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = crhyb.cr_solve(hyb, W, tol=1e-12, max_iter=50000, method="pcg", prec="mixed_bf16", inner_tol=1e-2,
                        raise_on_error=False)
    if st["status"] == 0:
        assert st["relres"] <= 1e-12
        U = torch.zeros(n, dtype=torch.float64, device="cuda")
        P = torch.zeros(hyb.mesh.ne, dtype=torch.float64, device="cuda")
        crhyb.cr_recover_up(hyb, W, U, P)
        assert rel(U.cpu().numpy(), ref["U"].ravel()) <= 1e-8
    else:
        assert st["status"] in (-4, -5) and st["status_name"] in ("CR_ERR_NOT_CONVERGED", "CR_ERR_BREAKDOWN")
        assert not (st["relres"] <= 1e-12)


def test_float_float_matches_fp64_iteration_count():
    """The float-float iteration follows the FP64 one: FF (48-bit values) needs
    at most a few per cent more iterations than FP64 PCG, the BF16-corrected
    values (about 32 bits) only slightly more."""
    case = make_case("2d_perturbed_37")
    _, _, hyb = gpu_setup(case)
    W = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    it = {}
    for prec in ("fp64", "ff", "ff_bf16"):
        W.zero_()
        st = crhyb.cr_solve(hyb, W, tol=1e-10, method="pcg", prec=prec)
        assert st["status"] == 0 and st["relres"] <= 1e-10
        it[prec] = st["iterations"]
    assert it["ff"] <= 1.05 * it["fp64"] + 2
    assert it["ff_bf16"] <= 1.25 * it["fp64"] + 2


@pytest.mark.parametrize("prec", ["fp64", "ff"])
def test_persistent_matches_multi_kernel_iteration(prec):
    """One persistent launch runs the same PCG as three launches per iteration:
    iteration counts agree to rounding (the dot products are summed in another
    order) and so do the solutions; a small chunk forces many relaunches."""
    case = make_case("2d_perturbed_37")
    _, _, hyb = gpu_setup(case)
    W0 = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    W1 = torch.zeros_like(W0)
    a = crhyb.cr_solve(hyb, W0, tol=1e-11, method="pcg", prec=prec)
    b = crhyb.cr_solve(hyb, W1, tol=1e-11, method="pcg", prec=prec, persistent=True, check_every=1)
    assert a["status"] == 0 and b["status"] == 0 and b["relres"] <= 1e-11
    assert abs(a["iterations"] - b["iterations"]) <= 0.02 * a["iterations"] + 2
    assert rel(W1.cpu().numpy(), W0.cpu().numpy()) <= 1e-9
    assert b["kernel_launches"] >= b["iterations"] // 64   # 64 iterations per launch with check_every=1


def test_persistent_tiny_mesh_limits_and_warm_start():
    coords, elems = synth.mesh2d_square(1)          # 2 triangles, 1 interior face, one tile
    mesh = crhyb.cr_mesh_load(coords, elems)
    hyb = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, 1.0, 10.0, np.ones((1, 2, 2))), keep_ff=True)
    for prec in ("fp64", "ff"):
        W = np.zeros(2)
        st = crhyb.cr_solve(hyb, W, tol=1e-14, prec=prec, persistent=True)
        assert st["status"] == 0 and st["relres"] <= 1e-13
    case = make_case("2d_perturbed_37")
    _, _, hyb = gpu_setup(case)
    W = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    st = crhyb.cr_solve(hyb, W, tol=1e-13, max_iter=7, prec="fp64", persistent=True, raise_on_error=False)
    assert st["status"] == -4 and st["iterations"] == 7
    st = crhyb.cr_solve(hyb, W, tol=1e-11, prec="ff", persistent=True)
    st2 = crhyb.cr_solve(hyb, W, tol=1e-10, prec="ff", persistent=True, use_x0=True)
    assert st2["status"] == 0 and st2["iterations"] <= 1


def test_persistent_barrier_timeout_is_reported(monkeypatch):
    """Failure detection without a fault: a block that leaves at once makes the
    other blocks' bounded grid-barrier waits run out; the solve returns
    CR_ERR_TIMEOUT and the context stays usable for the next solve."""
    case = make_case("2d_perturbed_37")
    _, _, hyb = gpu_setup(case)
    W = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
    monkeypatch.setenv("CRHYB_TEST_STALL_BLOCK", "0")
    with pytest.raises(crhyb.CrError) as ei:
        crhyb.cr_solve(hyb, W, tol=1e-10, prec="ff", persistent=True)
    assert ei.value.name == "CR_ERR_TIMEOUT"
    monkeypatch.delenv("CRHYB_TEST_STALL_BLOCK")
    st = crhyb.cr_solve(hyb, W, tol=1e-10, prec="ff", persistent=True)
    assert st["status"] == 0 and st["relres"] <= 1e-10


def test_second_rhs_and_host_buffers():
    case = make_case("2d_perturbed_37")
    coords, elems, nu, mu, conv, fbar, w = case
    _, system, hyb = gpu_setup(case)
    ref = pipeline.direct(coords, elems, nu, mu, fbar[1], conv, w, dense=True)
    n, ne = hyb.n, hyb.mesh.ne
    W = np.zeros(n)
    st = crhyb.cr_solve(hyb, W, rhs=1, tol=1e-13, method="pcg", prec="fp64")
    U, P = np.zeros(n), np.zeros(ne)
    crhyb.cr_recover_up(hyb, W, U, P, rhs=1)
    assert st["status"] == 0
    assert rel(U, ref["U"].ravel()) <= 1e-9
    assert rel(P, coupled.normalise_pressure(ref["P"], ref["geom"]["vol"])) <= 1e-9
    # warm start from the solution converges at once
    st2 = crhyb.cr_solve(hyb, W, rhs=1, tol=1e-10, method="pcg", prec="fp64", use_x0=True)
    assert st2["iterations"] <= 1


def test_k0_choice_does_not_change_normalised_pressure():
    case = make_case("cfg1")
    _, _, h0 = gpu_setup(case, k0=0)
    _, _, h1 = gpu_setup(case, k0=case[1].shape[0] - 1)
    _, _, U0, P0, _ = solve_and_recover(h0, 0, tol=1e-13)
    _, _, U1, P1, _ = solve_and_recover(h1, 0, tol=1e-13)
    assert rel(U1, U0) <= 1e-9 and rel(P1, P0) <= 1e-9


@pytest.mark.parametrize("dim", [2, 3])
def test_constant_source_closed_form(dim):
    """Section 4.1: a constant source gives U = 0 and P_K - P_{K_0} = f.(x_K - x_{K_0})."""
    coords, elems = synth.mesh2d_square(11, 0.2, 3) if dim == 2 else synth.mesh3d_kuhn(3)
    c = np.array([0.7, -1.3, 0.4][:dim])
    fbar = np.tile(c, (elems.shape[0], 1))[None].copy()
    mesh = crhyb.cr_mesh_load(coords, elems)
    hyb = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, 1.0, 100.0, fbar))
    W = np.zeros(hyb.n)
    crhyb.cr_solve(hyb, W, tol=1e-14)
    U, P = np.zeros(hyb.n), np.zeros(hyb.mesh.ne)
    crhyb.cr_recover_up(hyb, W, U, P, normalise_p=False)
    xK = coords[elems].mean(axis=1)
    assert np.abs(U).max() <= 1e-11
    assert np.abs(P - (xK - xK[0]) @ c).max() <= 1e-11


def test_tiny_mesh_and_error_paths():
    coords, elems = synth.mesh2d_square(1)          # 2 triangles, 1 interior face
    fbar = np.ones((1, 2, 2))
    mesh = crhyb.cr_mesh_load(coords, elems)
    assert mesh.nf == 1
    hyb = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, 1.0, 10.0, fbar))
    W = np.zeros(2)
    st = crhyb.cr_solve(hyb, W, tol=1e-14)
    assert st["status"] == 0
    with pytest.raises(crhyb.CrError) as ei:
        crhyb.cr_solve(hyb, W, rhs=3)
    assert ei.value.name == "CR_ERR_ARG"
    with pytest.raises(crhyb.CrError) as ei:
        crhyb.cr_solve(hyb, W, prec="mixed_bf16")      # BF16 values not kept
    assert ei.value.name == "CR_ERR_ARG"
    with pytest.raises(crhyb.CrError) as ei:
        crhyb.cr_solve(hyb, W, prec="ff")              # float-float values not kept
    assert ei.value.name == "CR_ERR_ARG"
    with pytest.raises(crhyb.CrError) as ei:
        crhyb.cr_solve(hyb, W, prec="ff", method="gmres")
    assert ei.value.name == "CR_ERR_ARG"
    with pytest.raises(crhyb.CrError) as ei:
        crhyb.cr_solve(hyb, W, prec="mixed", method="bicgstab")   # BiCGStab runs in FP64
    assert ei.value.name == "CR_ERR_ARG"
    # iteration limit
    case = make_case("2d_perturbed_37")
    _, _, hyb = gpu_setup(case)
    W = np.zeros(hyb.n)
    st = crhyb.cr_solve(hyb, W, tol=1e-13, max_iter=5, raise_on_error=False)
    assert st["status"] == -4 and st["iterations"] == 5
    # the E_K elimination at mu = 0 needs the independent set M_1 (the steady coupled
    # system itself does not: cr_solve_steady works on any mesh)
    steady = crhyb.cr_assemble_coupled(mesh, 1.0, 0.0, fbar)
    with pytest.raises(crhyb.CrError) as ei:
        crhyb.cr_hybridise(steady)
    assert ei.value.name == "CR_ERR_ARG"


@pytest.mark.parametrize("prec,persistent", [("mixed", False), ("ff", False), ("ff", True), ("fp64", True)])
def test_determinism(prec, persistent):
    case = make_case("2d_perturbed_37")
    _, _, hyb = gpu_setup(case)
    a = solve_and_recover(hyb, 0, tol=1e-12, prec=prec, persistent=persistent)
    b = solve_and_recover(hyb, 0, tol=1e-12, prec=prec, persistent=persistent)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[3], b[3]) and a[0] == b[0]


@pytest.mark.parametrize("opts", [dict(method="pcg", prec="fp64"), dict(method="pcg", prec="ff"),
                                  dict(method="pcg", prec="ff", persistent=True),
                                  dict(method="pcg", prec="fp64", persistent=True),
                                  dict(method="pcg", prec="mixed"), dict(method="gmres", prec="fp64"),
                                  dict(method="bicgstab", prec="fp64")],
                         ids=lambda o: "-".join(str(v) for v in o.values()))
def test_zero_source_gives_zero_solution(opts):
    """f = 0: S = 0, and every solver returns W = 0 at once (no division by ||S||)."""
    coords, elems = synth.mesh2d_square(7, 0.2, 5)
    case = (coords, elems, 1.0, 100.0, "none", np.zeros((1, elems.shape[0], 2)), None)
    mesh, _, hyb = gpu_setup(case)
    W = torch.ones(hyb.n, dtype=torch.float64, device="cuda")
    st = crhyb.cr_solve(hyb, W, tol=1e-10, **opts)
    assert st["status"] == 0 and st["iterations"] == 0 and st["relres"] == 0.0
    assert float(W.abs().max()) == 0.0
    U = torch.ones(hyb.n, dtype=torch.float64, device="cuda")
    P = torch.ones(mesh.ne, dtype=torch.float64, device="cuda")
    crhyb.cr_recover_up(hyb, W, U, P)
    assert float(U.abs().max()) == 0.0 and float(P.abs().max()) == 0.0


def test_zero_source_other_solvers():
    coords, elems = synth.mesh2d_square(7, 0.2, 5)
    zero = np.zeros((1, elems.shape[0], 2))
    case = (coords, elems, 1.0, 100.0, "none", zero, None)
    mesh, system, hyb = gpu_setup(case)
    pre = stokes_preconditioner(mesh, case)
    W = torch.ones(hyb.n, dtype=torch.float64, device="cuda")
    st = crhyb.cr_solve_preconditioned(hyb, pre, W, tol=1e-10)
    assert st["status"] == 0 and st["outer"] == 0 and float(W.abs().max()) == 0.0
    cpl = crhyb.cr_coupled_create(system)
    U = torch.ones(hyb.n, dtype=torch.float64, device="cuda")
    P = torch.ones(mesh.ne, dtype=torch.float64, device="cuda")
    st = crhyb.cr_solve_coupled(cpl, U, P, tol=1e-10, prec="fp64")
    assert st["status"] == 0 and st["iterations"] == 0
    assert float(U.abs().max()) == 0.0 and float(P.abs().max()) == 0.0
    batch = crhyb.cr_batch_create([hyb], prec="fp64")
    Wb = [torch.ones(hyb.n, dtype=torch.float64, device="cuda")]
    stb = crhyb.cr_solve_batched(batch, Wb, tol=1e-10)
    assert stb[0]["status"] == 0 and float(Wb[0].abs().max()) == 0.0


def test_user_stream_orders_inputs_and_outputs():
    """Every call orders its work after the caller's stream (the one given to
    cr_mesh_load) and the caller's stream after it: a source written late on
    that stream is the one the solve sees, and the recovered U can be read on
    it without a device-wide synchronisation."""
    case = make_case("2d_perturbed_37")
    coords, elems, nu, mu, conv, fbar, w = case
    ref = pipeline.direct(coords, elems, nu, mu, fbar[0], dense=True)
    s = torch.cuda.Stream()
    src = torch.from_numpy(np.ascontiguousarray(fbar)).cuda()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        fb = torch.zeros_like(src)
        torch.cuda._sleep(int(5e7))               # the source arrives late on the user stream
        fb.copy_(src)
        mesh = crhyb.cr_mesh_load(coords, elems, stream=s)
        hyb = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, nu, mu, fb), keep_fp32=False, keep_ff=True)
        W = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
        U = torch.zeros(hyb.n, dtype=torch.float64, device="cuda")
        P = torch.zeros(mesh.ne, dtype=torch.float64, device="cuda")
        crhyb.cr_solve(hyb, W, tol=1e-13, prec="ff", persistent=True)
        crhyb.cr_recover_up(hyb, W, U, P, normalise_p=True)
        Uc = U * 1.0                              # consumed on the user stream
    s.synchronize()
    assert rel(Uc.cpu().numpy(), ref["U"].ravel()) <= 1e-9
