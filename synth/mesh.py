"""Seeded simplicial meshes of the unit square and the unit cube.

Only vertex coordinates and vertex lists are produced here; faces, normals,
volumes and everything else the method derives from a mesh are computed
independently by the oracle and by the library.
"""

import numpy as np


def mesh2d_square(n, perturb=0.0, seed=0):
    """n x n squares of side h = 1/n, each split by its "/" diagonal.

    Square (i, j) with corners v00=(i,j), v10=(i+1,j), v11=(i+1,j+1),
    v01=(i,j+1) gives the triangles (v00, v10, v11) and (v00, v11, v01), in
    that order, squares taken row by row (i fastest).  When ``perturb`` > 0,
    every interior vertex moves by independent offsets drawn uniformly in
    [-perturb*h, perturb*h] for each coordinate (numpy default_rng(seed)).

    Returns (coords float64 [nv, 2], elems int32 [2 n^2, 3]).
    """
    n = int(n)
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 1.0 / n
    i, j = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
    coords = np.stack([i.ravel() * h, j.ravel() * h], axis=1).astype(np.float64)
    if perturb > 0.0:
        rng = np.random.default_rng(seed)
        off = rng.uniform(-perturb * h, perturb * h, size=coords.shape)
        interior = (i.ravel() > 0) & (i.ravel() < n) & (j.ravel() > 0) & (j.ravel() < n)
        coords[interior] += off[interior]
    vid = lambda a, b: a + (n + 1) * b  # noqa: E731
    si, sj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    si, sj = si.ravel(), sj.ravel()
    v00, v10, v11, v01 = vid(si, sj), vid(si + 1, sj), vid(si + 1, sj + 1), vid(si, sj + 1)
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    elems = np.empty((2 * n * n, 3), dtype=np.int32)
    elems[0::2] = t1
    elems[1::2] = t2
    _check_positive(coords, elems, oriented=True)
    return coords, elems


def mesh3d_kuhn(n):
    """n^3 cubes of side 1/n, each split into the 6 Kuhn tetrahedra.

    The 6 tetrahedra of a cube share its main diagonal v000-v111; tetrahedron
    number q follows the axis permutation q of (x, y, z) in lexicographic
    order: v000, v000 + e_a, v000 + e_a + e_b, v111.  Cubes are taken x
    fastest, then y, then z.

    Returns (coords float64 [(n+1)^3, 3], elems int32 [6 n^3, 4]).
    """
    n = int(n)
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 1.0 / n
    k, j, i = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
    coords = np.stack([i.ravel() * h, j.ravel() * h, k.ravel() * h], axis=1).astype(np.float64)
    vid = lambda a, b, c: a + (n + 1) * (b + (n + 1) * c)  # noqa: E731
    ck, cj, ci = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    tets = []
    for p in perms:
        pos = np.zeros((3, ci.size), dtype=np.int64)
        base = np.stack([ci, cj, ck])
        verts = [vid(*base)]
        for ax in p:
            pos[ax] += 1
            verts.append(vid(*(base + pos)))
        tets.append(np.stack(verts, axis=1))
    elems = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    _check_positive(coords, elems)
    return coords, elems


def batch_sizes(count=64, lo=8, hi=256, seed=2):
    """Mesh sizes n drawn log-uniformly in [lo, hi] and rounded (seeded)."""
    rng = np.random.default_rng(seed)
    return [int(v) for v in np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count)))]


def _check_positive(coords, elems, oriented=False):
    """Reject a generated mesh with a flat or folded simplex (a generator fault)."""
    X = coords[elems]
    J = X[:, 1:, :] - X[:, :1, :]
    det = np.linalg.det(J)
    tol = 1e-14 * (np.abs(J).max() ** J.shape[1])
    ok = (det > tol) if oriented else (np.abs(det) > tol)
    if not np.all(ok):
        raise AssertionError("generated mesh has a flat or folded simplex")
