"""Mesh topology for the CR scheme (Section 2, item 1; Section 3.2).

Faces are identified by their sorted vertex tuples; a face shared by two
simplices is interior (it carries the unknowns), a face of one simplex is
exterior (homogeneous Dirichlet, no unknown).  Local face l of a simplex is
the face opposite its local vertex l.
"""

import numpy as np


def build_faces(elems):
    """Interior faces and incidences of a simplicial mesh (Section 2, item 1).

    Returns a dict:
      face_vertices [nf, d]   sorted vertex tuple of each interior face, the
                              faces in lexicographic order of these tuples;
      elem_face [ne, d+1]     interior face index of local face l, or -1;
      face_elems [nf, 2]      the two simplices of each face, lower index first;
      face_local [nf, 2]      the local face index of the face in each of them;
      n_exterior              number of exterior faces.
    Raises ValueError when a face belongs to more than two simplices.
    """
    elems = np.asarray(elems, dtype=np.int64)
    ne, dp1 = elems.shape
    d = dp1 - 1
    keys = np.empty((ne, dp1, d), dtype=np.int64)
    for l in range(dp1):
        others = [m for m in range(dp1) if m != l]
        keys[:, l, :] = np.sort(elems[:, others], axis=1)
    flat = keys.reshape(-1, d)
    uniq, inverse, counts = np.unique(flat, axis=0, return_inverse=True, return_counts=True)
    inverse = inverse.ravel()
    if counts.max(initial=0) > 2:
        raise ValueError("a face belongs to more than two simplices")
    interior = counts == 2
    face_id = -np.ones(uniq.shape[0], dtype=np.int64)
    face_id[interior] = np.arange(int(interior.sum()))
    elem_face = face_id[inverse].reshape(ne, dp1)
    nf = int(interior.sum())
    face_elems = -np.ones((nf, 2), dtype=np.int64)
    face_local = -np.ones((nf, 2), dtype=np.int64)
    # incidences are visited in increasing element order, so slot 0 gets the lower index
    fill = np.zeros(nf, dtype=np.int64)
    for K in range(ne):
        for l in range(dp1):
            f = elem_face[K, l]
            if f >= 0:
                face_elems[f, fill[f]] = K
                face_local[f, fill[f]] = l
                fill[f] += 1
    return {
        "d": d,
        "ne": ne,
        "nf": nf,
        "face_vertices": uniq[interior],
        "elem_face": elem_face,
        "face_elems": face_elems,
        "face_local": face_local,
        "n_exterior": int((counts == 1).sum()),
    }


def owner_signs(topo):
    """Diagonal of C_K per local face (Section 3.2, Eq. 12).

    C_{K,sigma} = +1 when K is the lower-index simplex of the interior face
    sigma (its owner) and -1 for the other simplex, so C_K + C_L = 0; the
    entry of an exterior face is 0 (it carries no unknown).
    """
    ne, dp1 = topo["elem_face"].shape
    C = np.zeros((ne, dp1))
    fe, fl = topo["face_elems"], topo["face_local"]
    C[fe[:, 0], fl[:, 0]] = 1.0
    C[fe[:, 1], fl[:, 1]] = -1.0
    return C


def neighbours(topo):
    """Face-adjacency lists of the simplices (two simplices sharing a face)."""
    ne = topo["ne"]
    nb = [[] for _ in range(ne)]
    for K, L in topo["face_elems"]:
        nb[K].append(int(L))
        nb[L].append(int(K))
    return nb


def maximal_independent_set(topo):
    """M_1 for the mu = 0 choice of E_K (Section 3.2, item 7).

    M_1 is a maximal set of simplices no two of which share a face, built
    greedily in increasing simplex index; M_2 (all other simplices) is then
    exactly the set of neighbours of M_1.  Returns a bool array [ne].
    """
    nb = neighbours(topo)
    in_m1 = np.zeros(topo["ne"], dtype=bool)
    for K in range(topo["ne"]):
        if not any(in_m1[L] for L in nb[K]):
            in_m1[K] = True
    return in_m1
