"""The allocation-free residual entry point, cr_residual_noalloc.

Some callers cannot allocate device memory: a host application that owns
every allocation through its own pool, code that must not take the implicit
device synchronisation of cudaMalloc/cudaFree on its hot path, or a checker
that must leave the device's memory exactly as it found it.  For them
cr_residual_noalloc computes r = b - G x and ||r||^2, ||b||^2 with its only
scratch in a fixed device array inside the library.

These tests compare it, on two calls in a row (the scratch keeps the previous
call's contents), with the library's allocating entry points (cr_solve's FP64
residual of its returned W, cr_apply_G) and with the oracle's own G and S
(assembled on the CPU from the paper's formulas, in the same face order).
Tolerance: 1e-12 relative to the size of b (the same FP64 sums in another
order).  They also check that a column index outside [0, nf) is rejected
without leaving a stale counter behind, and a mesh of several hundred tiles,
whose per-tile partial sums the last block accumulates with a stride.  The
file name makes pytest collect it last.
"""

import numpy as np
import pytest

import synth
from oracle import pipeline, hybrid
from paper_2101_03777_gb300 import crhyb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(n=37, nrhs=2):
    p = synth.config_problem("cfg2", n=n, nrhs=nrhs)
    mesh = crhyb.cr_mesh_load(p["coords"], p["elems"])
    fbar = torch.from_numpy(p["fbar"]).cuda()
    hyb = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, p["nu"], p["mu"], fbar))
    cols, vals, S = crhyb.cr_hybrid_export(hyb)
    return p, hyb, torch.from_numpy(cols).cuda(), torch.from_numpy(vals).cuda(), torch.from_numpy(S).cuda()


def test_noalloc_residual_matches_allocating_entry_points():
    _, hyb, cols, vals, S = _setup()
    d, nf, n = hyb.mesh.dim, hyb.mesh.nf, hyb.n
    scale = float(S.abs().max())
    for call, rhs in enumerate((0, 1)):
        b = S[rhs].reshape(-1).contiguous()
        W = torch.zeros(n, dtype=torch.float64, device="cuda")
        st = crhyb.cr_solve(hyb, W, rhs=rhs, tol=1e-11, method="pcg", prec="fp64")
        # the existing entry points: G x by cr_apply_G, relres from cr_solve
        GW = torch.empty_like(W)
        crhyb.cr_apply_G(hyb, W, GW)
        r_ref = b - GW
        r = torch.full_like(W, float("nan"))
        norms = crhyb.cr_residual_noalloc(d, nf, cols, vals, b, W, r)
        assert torch.isfinite(r).all()
        assert float((r - r_ref).abs().max()) <= 1e-12 * scale, f"call {call}"
        assert abs(norms[1] - float(b @ b)) <= 1e-12 * float(b @ b)
        rel = np.sqrt(norms[0] / norms[1])
        assert abs(rel - st["relres"]) <= 1e-12 * scale / np.sqrt(norms[1]) * np.sqrt(n), f"call {call}"
        # x = 0 gives r = b exactly
        r0 = torch.empty_like(W)
        n0 = crhyb.cr_residual_noalloc(d, nf, cols, vals, b, torch.zeros_like(W), r0)
        assert torch.equal(r0, b) and n0[0] == n0[1]


def test_noalloc_residual_matches_the_oracle_G():
    """r = S - G x with G and S the oracle's (Section 3.2, items 4 and 5), x seeded."""
    p, hyb, cols, vals, _ = _setup(n=24, nrhs=1)
    d, nf = hyb.mesh.dim, hyb.mesh.nf
    topo, _, A_K, D_K, R_K = pipeline.setup(p["coords"], p["elems"], p["nu"], p["mu"], p["fbar"][0])
    h = hybrid.hybridise(topo, A_K, D_K, R_K, p["mu"])
    Go, So = h["G"], h["S"]
    rng = np.random.default_rng(7)
    for call in range(2):
        x = rng.standard_normal(nf * d)
        r_or = So - Go @ x
        b = torch.from_numpy(So).cuda()
        r = torch.empty_like(b)
        norms = crhyb.cr_residual_noalloc(d, nf, cols, vals, b, torch.from_numpy(x).cuda(), r)
        scale = float(np.abs(So).max() + np.abs(Go @ x).max())
        assert np.abs(r.cpu().numpy() - r_or).max() <= 1e-12 * scale, f"call {call}"
        assert abs(norms[0] - r_or @ r_or) <= 1e-11 * (r_or @ r_or)
        assert abs(norms[1] - So @ So) <= 1e-12 * (So @ So)


def test_noalloc_residual_rejects_out_of_range_columns_then_recovers():
    _, hyb, cols, vals, S = _setup(n=16, nrhs=1)
    d, nf, n = hyb.mesh.dim, hyb.mesh.nf, hyb.n
    b = S[0].reshape(-1).contiguous()
    x = torch.linspace(-1.0, 1.0, n, dtype=torch.float64, device="cuda")
    for bad_value in (nf, -1):
        bad = cols.clone()
        bad[1, nf // 2] = bad_value
        with pytest.raises(crhyb.CrError) as ei:
            crhyb.cr_residual_noalloc(d, nf, bad, vals, b, x, torch.empty_like(b))
        assert ei.value.name == "CR_ERR_ARG" and "out of range" in str(ei.value)
        # the next unmodified call starts from clean counters and matches cr_apply_G
        Gx = torch.empty_like(x)
        crhyb.cr_apply_G(hyb, x, Gx)
        r = torch.empty_like(b)
        norms = crhyb.cr_residual_noalloc(d, nf, cols, vals, b, x, r)
        ref = b - Gx
        assert float((r - ref).abs().max()) <= 1e-12 * float(b.abs().max() + Gx.abs().max())
        assert abs(norms[0] - float(ref @ ref)) <= 1e-11 * float(ref @ ref)


def test_noalloc_residual_on_several_hundred_tiles():
    """cfg2 shape at 200 x 200 squares: 119,600 face rows, 468 tiles, so the last
    block accumulates the per-tile partials with a stride over its threads."""
    _, hyb, cols, vals, S = _setup(n=200, nrhs=1)
    d, nf, n = hyb.mesh.dim, hyb.mesh.nf, hyb.n
    assert (nf + 255) // 256 > 256
    b = S[0].reshape(-1).contiguous()
    g = torch.Generator(device="cuda").manual_seed(11)
    for call in range(2):
        x = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
        Gx = torch.empty_like(x)
        crhyb.cr_apply_G(hyb, x, Gx)
        ref = b - Gx
        r = torch.empty_like(b)
        norms = crhyb.cr_residual_noalloc(d, nf, cols, vals, b, x, r)
        assert float((r - ref).abs().max()) <= 1e-12 * float(b.abs().max() + Gx.abs().max()), f"call {call}"
        assert abs(norms[0] - float(ref @ ref)) <= 1e-11 * float(ref @ ref)
        assert abs(norms[1] - float(b @ b)) <= 1e-12 * float(b @ b)


def test_noalloc_residual_rejects_sizes_beyond_its_scratch():
    _, hyb, cols, vals, S = _setup()
    big = crhyb.cr_residual_noalloc_max_rows() + 1
    with pytest.raises(crhyb.CrError) as ei:
        crhyb.cr_residual_noalloc(2, big, cols, vals, S[0].reshape(-1), S[0].reshape(-1), None, check_sizes=False)
    assert ei.value.name == "CR_ERR_ARG" and "scratch" in str(ei.value)
