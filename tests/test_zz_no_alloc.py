"""The allocation-free residual entry point, cr_residual_noalloc.

Some callers cannot allocate device memory: a host application that owns
every allocation through its own pool, code that must not take the implicit
device synchronisation of cudaMalloc/cudaFree on its hot path, or a checker
that must leave the device's memory exactly as it found it.  For them
cr_residual_noalloc computes r = b - G x and ||r||^2, ||b||^2 with its only
scratch in a fixed device array inside the library.

This test compares it, on two calls in a row (the scratch keeps the previous
call's contents), with the library's allocating entry points: cr_solve's FP64
residual of its returned W and cr_apply_G.  Tolerance: 1e-12 relative to the
size of b (same FP64 sums in a different order).  The file name makes pytest
collect it last.
"""

import numpy as np
import pytest

import synth
from paper_2101_03777_gb300 import crhyb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup():
    p = synth.config_problem("cfg2", n=37, nrhs=2)
    mesh = crhyb.cr_mesh_load(p["coords"], p["elems"])
    fbar = torch.from_numpy(p["fbar"]).cuda()
    hyb = crhyb.cr_hybridise(crhyb.cr_assemble_coupled(mesh, p["nu"], p["mu"], fbar))
    cols, vals, S = crhyb.cr_hybrid_export(hyb)
    return hyb, torch.from_numpy(cols).cuda(), torch.from_numpy(vals).cuda(), torch.from_numpy(S).cuda()


def test_noalloc_residual_matches_allocating_entry_points():
    hyb, cols, vals, S = _setup()
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


def test_noalloc_residual_rejects_sizes_beyond_its_scratch():
    hyb, cols, vals, S = _setup()
    big = crhyb.cr_residual_noalloc_max_rows() + 1
    with pytest.raises(crhyb.CrError) as ei:
        crhyb.cr_residual_noalloc(2, big, cols, vals, S[0].reshape(-1), S[0].reshape(-1), None, check_sizes=False)
    assert ei.value.name == "CR_ERR_ARG" and "scratch" in str(ei.value)
