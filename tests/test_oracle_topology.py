"""Pins for the oracle's mesh topology (Section 2, item 1; Section 3.2).

Closed-form face counts of the structured meshes, incidence consistency,
the C_K sign rule (C_K + C_L = 0, Eq. 12) and the maximal independent set
used for E_K when mu = 0 (Section 3.2, item 7).
"""

import numpy as np
import pytest

import synth
from oracle import topology


@pytest.mark.parametrize("n", [1, 2, 5, 16])
def test_2d_face_counts(n):
    # 2 n^2 triangles: 3 (2n^2) = 2 F_int + F_ext, F_ext = 4n
    _, elems = synth.mesh2d_square(n)
    t = topology.build_faces(elems)
    assert t["nf"] == 3 * n * n - 2 * n
    assert t["n_exterior"] == 4 * n


@pytest.mark.parametrize("n", [1, 2, 4])
def test_3d_face_counts(n):
    # 6 n^3 tetrahedra: 4 (6 n^3) = 2 F_int + F_ext, F_ext = 12 n^2
    _, elems = synth.mesh3d_kuhn(n)
    t = topology.build_faces(elems)
    assert t["nf"] == 12 * n ** 3 - 6 * n ** 2
    assert t["n_exterior"] == 12 * n * n


@pytest.mark.parametrize("dim", [2, 3])
def test_incidence_consistency(dim):
    _, elems = synth.mesh2d_square(4, 0.2, 1) if dim == 2 else synth.mesh3d_kuhn(2)
    t = topology.build_faces(elems)
    fe, fl, fv = t["face_elems"], t["face_local"], t["face_vertices"]
    assert np.all(fe[:, 0] < fe[:, 1])
    for f in range(t["nf"]):
        for s in range(2):
            K, l = fe[f, s], fl[f, s]
            assert t["elem_face"][K, l] == f
            verts = sorted(int(v) for m, v in enumerate(elems[K]) if m != l)
            assert verts == list(fv[f])
    # lexicographic order of the vertex tuples
    keys = [tuple(r) for r in fv]
    assert keys == sorted(keys)
    # every local face slot is either an interior face or exterior
    assert (t["elem_face"] >= 0).sum() == 2 * t["nf"]


def test_owner_signs():
    _, elems = synth.mesh2d_square(4)
    t = topology.build_faces(elems)
    C = topology.owner_signs(t)
    fe, fl = t["face_elems"], t["face_local"]
    assert np.all(C[fe[:, 0], fl[:, 0]] + C[fe[:, 1], fl[:, 1]] == 0)
    assert np.all(np.abs(C[t["elem_face"] >= 0]) == 1)
    assert np.all(C[t["elem_face"] < 0] == 0)


@pytest.mark.parametrize("dim", [2, 3])
def test_mis_is_maximal_independent(dim):
    _, elems = synth.mesh2d_square(6, 0.2, 2) if dim == 2 else synth.mesh3d_kuhn(2)
    t = topology.build_faces(elems)
    m1 = topology.maximal_independent_set(t)
    fe = t["face_elems"]
    assert not np.any(m1[fe[:, 0]] & m1[fe[:, 1]])          # independent
    nb = topology.neighbours(t)
    for K in range(t["ne"]):                                 # maximal: M_2 = neighbours of M_1
        if not m1[K]:
            assert any(m1[L] for L in nb[K])


def test_face_in_three_simplices_is_rejected():
    elems = np.array([[0, 1, 2], [0, 1, 3], [0, 1, 4]], dtype=np.int32)
    with pytest.raises(ValueError):
        topology.build_faces(elems)
