"""Oracle truths for the full-size U/P parity tests (test infrastructure).

Each function runs the CPU FP64 oracle on one problem and returns U [nf*d]
and P [ne] normalised to zero mean (Section 2, item 5), the quantities the
GPU path is compared with.  They run in spawned worker processes while the
GPU solves run, so every input is rebuilt here from the seeded generators.

* 2D: the oracle's hybrid method with a direct solve of G W = S (SciPy's
  sparse LU), then the element-wise recovery (Section 3.2): the method
  reaches the coupled solution exactly, so this is the coupled solution up to
  rounding (the oracle's hybridisation is pinned to the coupled direct solve
  on small meshes).
* 3D: the oracle's Jacobi-PCG on G W = S to a relative residual of 1e-12, then
  the recovery (a direct factorisation of the 3D G at this size does not fit
  the test's time).  On 2D meshes the recovered U of a PCG solve to 1e-13 is
  within 1.5e-13 of the direct solve's (128x128), so 1e-12 leaves a margin of
  about 1e3 below the 1e-9 parity tolerance.
"""

import numpy as np
import scipy.sparse.linalg as spla

import synth
from oracle import coupled, hybrid, krylov, pipeline, topology


def _up(h, topo, geom, W, R_K=None):
    U, P, _ = hybrid.recover(h, topo, W, R_K)
    return U, coupled.normalise_pressure(P, geom["vol"])


def stokes_2d(n, nrhs=1):
    """cfg2 family (perturbed 2D squares, nu = 1, mu = 1000) at n x n: list of (U, P) per rhs."""
    p = synth.config_problem("cfg2", n=n, nrhs=nrhs)
    out = []
    lu = None
    for r in range(nrhs):
        topo, geom, A_K, D_K, R_K = pipeline.setup(p["coords"], p["elems"], p["nu"], p["mu"], p["fbar"][r])
        h = hybrid.hybridise(topo, A_K, D_K, R_K, p["mu"])
        if lu is None:
            lu = spla.splu(h["G"].tocsc())
        out.append(_up(h, topo, geom, lu.solve(h["S"])))
    return out


def stokes_3d(n, rtol=1e-12):
    """cfg3 family (3D Kuhn cubes, nu = 1, mu = 1000) at n^3: (U, P, oracle PCG iterations)."""
    p = synth.config_problem("cfg3", n=n)
    topo, geom, A_K, D_K, R_K = pipeline.setup(p["coords"], p["elems"], p["nu"], p["mu"], p["fbar"][0])
    h = hybrid.hybridise(topo, A_K, D_K, R_K, p["mu"])
    W, it, _ = krylov.pcg(h["G"], h["S"], krylov.jacobi(h["G"]), rtol=rtol)
    U, P = _up(h, topo, geom, W)
    return U, P, it


def batch_problem(k, count=64, nrhs=4, lo=8, hi=256, seed=2):
    """Problem k of the batched workload (perturbed 2D squares), every rhs: list of (U, P)."""
    q = synth.batch_problems(count=count, nrhs=nrhs, lo=lo, hi=hi, seed=seed)[k]
    out = []
    lu = None
    for r in range(nrhs):
        topo, geom, A_K, D_K, R_K = pipeline.setup(q["coords"], q["elems"], q["nu"], q["mu"], q["fbar"][r])
        h = hybrid.hybridise(topo, A_K, D_K, R_K, q["mu"])
        if lu is None:
            lu = spla.splu(h["G"].tocsc())
        out.append(_up(h, topo, geom, lu.solve(h["S"])))
    return out


def newton_2d(n, nu=0.01, mu=1000.0):
    """A transient Newton step (cfg5 family, unperturbed 2D squares, linearised about the
    seeded stream-function field) at n x n, direct solve of the nonsymmetric G: (U, P)."""
    coords, elems = synth.mesh2d_square(n)
    modes = synth.fourier_modes(2, 1)
    fbar = synth.element_means(lambda x: synth.fourier_force(x, modes), coords, elems, order=3)
    t = topology.build_faces(elems)
    w = synth.stream_velocity(coords[t["face_vertices"]].mean(axis=1), seed=3)
    topo, geom, A_K, D_K, R_K = pipeline.setup(coords, elems, nu, mu, fbar, "newton", w)
    h = hybrid.hybridise(topo, A_K, D_K, R_K, mu)
    W = spla.spsolve(h["G"].tocsc(), h["S"])
    return _up(h, topo, geom, W)


def newton_2d_inputs(n):
    """The GPU side's inputs of newton_2d: coords, elems, fbar [1, ne, 2], w [nf, 2]."""
    coords, elems = synth.mesh2d_square(n)
    modes = synth.fourier_modes(2, 1)
    fbar = synth.element_means(lambda x: synth.fourier_force(x, modes), coords, elems, order=3)[None]
    t = topology.build_faces(elems)
    w = synth.stream_velocity(coords[t["face_vertices"]].mean(axis=1), seed=3)
    return coords, elems, np.ascontiguousarray(fbar), np.ascontiguousarray(w)
