"""Algebraic hybridisation of Eq. 10, step by step (Section 3.2).

The hybrid method: (1) compute G and S, (2) solve G W = S, (3) recover P
and U element by element (Section 3.2, closing list).  Every element
quantity here is an explicit dense matrix of the simplex's (d+1) d local
unknowns; rows and columns of exterior faces are inert (zero in A_K, D_K,
R_K; identity in the padded Â_K so that its inverse restricted to the
interior unknowns is the inverse of the interior block).
"""

import numpy as np
import scipy.sparse as sp

from . import elements, topology


def e_diagonals(topo, A_K, mu, lam_scale=2.0):
    """Diagonals of E_K (Section 3.2, items 6 and 7).

    mu > 0: E_K = 0.
    mu = 0: M_1 = maximal independent set (greedy, increasing index); for
      K in M_1, E_K = -lambda_K Id with lambda_K = lam_scale * ||A_K||_inf,
      the row-sum norm, which exceeds the modulus of every eigenvalue of A_K;
      for K in M_2 and a face shared with L in M_1, (E_K)_{sigma sigma} =
      +lambda_L, and 0 on the other faces.  Thus E_K + E_L = 0 (Eq. 11).
    Returns (E [ne, (d+1) d], in_m1 or None, lam [ne] or None).
    """
    ne, nl, _ = A_K.shape
    d = topo["d"]
    E = np.zeros((ne, nl))
    if mu > 0.0:
        return E, None, None
    mask = elements.interior_mask(topo)
    in_m1 = topology.maximal_independent_set(topo)
    lam = lam_scale * np.abs(A_K).sum(axis=2).max(axis=1)
    E[in_m1] = -lam[in_m1, None] * mask[in_m1]
    fe, fl = topo["face_elems"], topo["face_local"]
    for f in range(topo["nf"]):
        K, L = fe[f]
        lk, ll = fl[f]
        if in_m1[K]:
            E[L, ll * d:(ll + 1) * d] = lam[K]
        if in_m1[L]:
            E[K, lk * d:(lk + 1) * d] = lam[L]
    return E, in_m1, lam


def hybridise(topo, A_K, D_K, R_K, mu, k0=0, lam_scale=2.0):
    """G and S of Section 3.2, item 4, with G = sum_K H_K G_K H_K^t (item 5).

    Â_K = A_K + E_K;  B_K = D_K^t Â_K^{-1} D_K;
    G_K = C_K (Â_K^{-1} - Â_K^{-1} D_K D_K^t Â_K^{-1} / B_K) C_K  (K != K_0),
    G_{K_0} = C_{K_0} Â_{K_0}^{-1} C_{K_0};
    S = sum_K H_K C_K M_K R_K, M_K being the bracket of G_K.
    R_K may be [ne, nl] or [nrhs, ne, nl].
    """
    ne, nl, _ = A_K.shape
    d = topo["d"]
    mask = elements.interior_mask(topo)
    E, in_m1, lam = e_diagonals(topo, A_K, mu, lam_scale)
    Ahat = A_K + E[:, :, None] * np.eye(nl)[None]
    pad = np.where(mask, 0.0, 1.0)
    Ainv = np.linalg.inv(Ahat + pad[:, :, None] * np.eye(nl)[None])
    Ainv = Ainv * mask[:, :, None] * mask[:, None, :]
    Cv = np.repeat(topology.owner_signs(topo), d, axis=1)
    u = np.einsum("kab,kb->ka", Ainv, D_K)          # Â^{-1} D
    wt = np.einsum("ka,kab->kb", D_K, Ainv)         # D^t Â^{-1}
    B = np.einsum("ka,ka->k", D_K, u)
    M = Ainv - np.einsum("ka,kb->kab", u, wt) / np.where(B == 0.0, 1.0, B)[:, None, None]
    M[k0] = Ainv[k0]
    GK = Cv[:, :, None] * M * Cv[:, None, :]
    dofs = elements.local_dofs(topo)
    N = topo["nf"] * d
    rows = np.repeat(dofs, nl, axis=1).ravel()
    cols = np.tile(dofs, (1, nl)).ravel()
    keep = (rows >= 0) & (cols >= 0)
    G = sp.coo_matrix((GK.reshape(ne, -1).ravel()[keep], (rows[keep], cols[keep])),
                      shape=(N, N)).tocsr()
    R3 = R_K[None] if R_K.ndim == 2 else R_K
    S = np.zeros((R3.shape[0], N))
    kp = dofs >= 0
    for j in range(R3.shape[0]):
        SK = Cv * np.einsum("kab,kb->ka", M, R3[j])
        np.add.at(S[j], dofs[kp], SK[kp])
    return {"G": G, "S": S if R_K.ndim == 3 else S[0], "GK": GK, "Ainv": Ainv, "B": B,
            "Cv": Cv, "E": E, "in_m1": in_m1, "lam": lam, "D_K": D_K, "R_K": R_K,
            "dofs": dofs, "k0": k0, "d": d}


def recover(hyb, topo, W, R_K=None):
    """P and U from W (Section 3.2, items 2 and 4).

    With y = R_K - C_K W_K:  P_K = D_K^t Â_K^{-1} y / B_K (K != K_0),
    P_{K_0} = 0;  Û_K = Â_K^{-1} (y - D_K P_K);  U_sigma = Û_{K,sigma}
    taken from the owner, Û_{K,sigma} = Û_{L,sigma} holding by Eq. 15.
    Returns (U [nf*d], P [ne], jump = max |Û_K - Û_L| over faces).
    """
    R_K = hyb["R_K"] if R_K is None else R_K
    dofs, Cv, Ainv, D_K, B, k0 = (hyb[k] for k in ("dofs", "Cv", "Ainv", "D_K", "B", "k0"))
    d = hyb["d"]
    Wl = np.where(dofs >= 0, W[np.maximum(dofs, 0)], 0.0)
    y = R_K - Cv * Wl
    Ay = np.einsum("kab,kb->ka", Ainv, y)
    P = np.einsum("ka,ka->k", D_K, Ay) / np.where(B == 0.0, 1.0, B)
    P[k0] = 0.0
    Uhat = Ay - np.einsum("kab,kb->ka", Ainv, D_K) * P[:, None]
    fe, fl = topo["face_elems"], topo["face_local"]
    nf = topo["nf"]
    own = Uhat.reshape(-1, d + 1, d)[fe[:, 0], fl[:, 0]]
    oth = Uhat.reshape(-1, d + 1, d)[fe[:, 1], fl[:, 1]]
    jump = float(np.abs(own - oth).max()) if nf else 0.0
    return own.reshape(nf * d), P, jump
