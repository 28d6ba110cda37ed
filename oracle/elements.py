"""Element geometry and element matrices of the CR scheme (Sections 2 and 3.1).

Arrays are batched over simplices: X [ne, d+1, d] holds the vertices; local
face l is opposite local vertex l.  Velocity unknowns of a simplex are
ordered (l, i) -> l*d + i (face-major, component fastest).
"""

import math

import numpy as np


def geometry(coords, elems):
    """|K|, x_K, x_sigma and a_{K,sigma} = |sigma| n_{K,sigma} (Section 2, item 1).

    The outward normal is taken from the face itself (edge normal in 2D,
    half the cross product of two edges in 3D), oriented away from the
    opposite vertex.  Returns a dict of arrays.
    """
    X = np.asarray(coords, dtype=np.float64)[np.asarray(elems)]
    ne, dp1, d = X.shape
    J = X[:, 1:, :] - X[:, :1, :]
    vol = np.abs(np.linalg.det(J)) / math.factorial(d)
    xK = X.mean(axis=1)
    xs = (X.sum(axis=1)[:, None, :] - X) / d
    a = np.empty((ne, dp1, d))
    for l in range(dp1):
        P = X[:, [m for m in range(dp1) if m != l], :]
        if d == 2:
            t = P[:, 1] - P[:, 0]
            nrm = np.stack([t[:, 1], -t[:, 0]], axis=1)          # length |sigma|
        else:
            nrm = 0.5 * np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])  # length |sigma|
        out = np.einsum("kd,kd->k", xs[:, l] - X[:, l], nrm) > 0.0
        a[:, l] = np.where(out[:, None], nrm, -nrm)
    return {"X": X, "vol": vol, "xK": xK, "xs": xs, "a": a, "d": d}


def cr_gradients(geom):
    """Gradients of the CR basis functions on each simplex (Section 2, item 1).

    phi_sigma restricted to K is the affine function whose mean over face
    tau equals delta_{sigma tau}; the mean of an affine function over a face
    is its value at the face centroid, so its coefficients solve
    [1, x_tau] c = e_sigma.  Returns grad [ne, d+1 (sigma), d].
    """
    xs = geom["xs"]
    ne, dp1, d = xs.shape
    M = np.concatenate([np.ones((ne, dp1, 1)), xs], axis=2)   # rows: faces tau
    coef = np.linalg.inv(M)                                  # column sigma = phi_sigma
    return np.transpose(coef[:, 1:, :], (0, 2, 1))


def local_S(geom, nu, mu):
    """S_K over all d+1 local faces (Section 3.1; Section 2, items 2-3).

    (S_K)_{sigma sigma'} = nu |K| grad phi_sigma . grad phi_sigma'
                           + mu |D_{K,sigma}| delta_{sigma sigma'},
    where the lumped mass uses the co-volume D_{K,sigma}, the cone on sigma
    with apex x_K, of measure |K|/(d+1); in 2D this is also the exact CR
    mass matrix, which is diagonal.  Rows of exterior faces are kept here;
    the caller restricts to interior faces.
    """
    g = cr_gradients(geom)
    vol = geom["vol"]
    d = geom["d"]
    S = nu * vol[:, None, None] * np.einsum("kad,kbd->kab", g, g)
    S += (mu * vol / (d + 1))[:, None, None] * np.eye(d + 1)[None]
    return S


def local_A(S):
    """A_K = S_K (x) Id_d in the (l, i) -> l*d + i ordering (Section 3.1, b_h = 0)."""
    ne, dp1, _ = S.shape
    d = dp1 - 1
    return np.einsum("kab,ij->kaibj", S, np.eye(d)).reshape(ne, dp1 * d, dp1 * d)


def local_D(geom):
    """D_K with (D_K)_{i,sigma} = -a^(i)_{K,sigma} (Section 3.1); [ne, (d+1) d]."""
    a = geom["a"]
    return -a.reshape(a.shape[0], -1)


def local_R(geom, fbar):
    """R_K from the RT reconstruction of the source (Eq. 8, Section 3.1).

    (R_K)_{i,sigma} = a^(i)_{K,sigma} fbar_K . (x_sigma - x_K); fbar [ne, d].
    Returns [ne, (d+1) d].
    """
    a, xs, xK = geom["a"], geom["xs"], geom["xK"]
    rho = np.einsum("kd,kld->kl", fbar, xs - xK[:, None, :])
    return (a * rho[:, :, None]).reshape(a.shape[0], -1)


def local_R_previous(topo, geom, mu, u_prev):
    """Implicit Euler with mu = 1/dt (Section 2, the transient problem with the
    time derivative discretised by one backward step): the mass term of S_K,
    mu |K|/(d+1) per interior face (Section 3.1, the lumped mass), applied to
    the previous time level and moved to the right-hand side.

    (R_K)_{i,sigma} += mu |K|/(d+1) u^n_{sigma,i}; u_prev [nf, d] or [nf*d].
    Returns [ne, (d+1) d], zero on exterior faces.
    """
    d = topo["d"]
    ef = topo["elem_face"]
    U = np.asarray(u_prev, dtype=np.float64).reshape(-1, d)
    loc = np.where((ef >= 0)[:, :, None], U[np.maximum(ef, 0)], 0.0)
    mass = mu * geom["vol"] / (d + 1)                     # [ne]
    return (mass[:, None, None] * loc).reshape(ef.shape[0], -1)


def interior_mask(topo):
    """[ne, (d+1) d] mask of the local unknowns that live on interior faces."""
    m = topo["elem_face"] >= 0
    d = topo["d"]
    return np.repeat(m, d, axis=1)


def local_dofs(topo):
    """Global unknown index (face*d + i) of each local unknown, -1 on exterior faces."""
    ef = topo["elem_face"]
    d = topo["d"]
    idx = ef[:, :, None] * d + np.arange(d)[None, None, :]
    idx[ef < 0] = -1
    return idx.reshape(ef.shape[0], -1)
