"""The co-volume convection form b_h of Eq. 9 (Section 2, item 6).

For a simplex K with local face velocities U_l (zero on exterior faces,
homogeneous Dirichlet):

  F_{l m}(u) = (U_l + U_m - (1/(d+1)) sum_n U_n) . (a_m - a_l)/(d+1),
  c_l(u)     = 1/2 sum_{m != l} F_{l m}(u) (U_m - U_l),

c_l being the coefficient of the test value V_l in b_h restricted to K.
c is quadratic in u; its Newton derivative at w and its Oseen (Picard)
linearisation are given below.  Local unknown order: (l, i) -> l*d + i.
"""

import numpy as np


def fluxes(U, a):
    """F_{l m}(u) for every ordered pair of local faces; U, a [ne, d+1, d] -> [ne, d+1, d+1]."""
    dp1 = U.shape[1]
    Ubar = U.mean(axis=1, keepdims=True)
    base = U[:, :, None, :] + U[:, None, :, :] - Ubar[:, :, None, :]      # [k, l, m, d]
    g = (a[:, None, :, :] - a[:, :, None, :]) / dp1                       # (a_m - a_l)/(d+1)
    return np.einsum("klmd,klmd->klm", base, g)


def element_convection(U, a):
    """c_l(u) for each simplex: [ne, d+1, d] (Eq. 9, second form)."""
    F = fluxes(U, a)
    dU = U[:, None, :, :] - U[:, :, None, :]                              # U_m - U_l
    return 0.5 * np.einsum("klm,klmd->kld", F, dU)                        # m = l term is 0


def bh_pairs(U, V, a):
    """b_h(u, v) summed over simplices from the unordered-pair form of Eq. 9."""
    F = fluxes(U, a)
    dp1 = U.shape[1]
    total = 0.0
    for l in range(dp1):
        for m in range(l + 1, dp1):
            total += np.sum(F[:, l, m] * np.einsum("kd,kd->k", U[:, m] - U[:, l],
                                                    0.5 * (V[:, l] + V[:, m])))
    return total


def newton_jacobian(W, a):
    """d c_l / d U_n at u = w, as a [ne, (d+1) d, (d+1) d] matrix.

    Differentiating c_l = 1/2 sum_{m != l} F_{lm}(u) (U_m - U_l), with
    d F_{lm} / d U_n = g_{lm}^T (delta_{nl} + delta_{nm} - 1/(d+1)):
      1/2 sum_{m != l} [ (W_m - W_l) g_{lm}^T (delta_{nl} + delta_{nm} - 1/(d+1))
                         + F_{lm}(w) (delta_{nm} - delta_{nl}) Id ].
    """
    ne, dp1, d = W.shape
    F = fluxes(W, a)
    g = (a[:, None, :, :] - a[:, :, None, :]) / dp1
    Jm = np.zeros((ne, dp1, d, dp1, d))
    eye = np.eye(d)
    for l in range(dp1):
        for m in range(dp1):
            if m == l:
                continue
            outer = np.einsum("ki,kj->kij", W[:, m] - W[:, l], g[:, l, m])
            for n in range(dp1):
                coef = (1.0 if n == l else 0.0) + (1.0 if n == m else 0.0) - 1.0 / dp1
                Jm[:, l, :, n, :] += 0.5 * coef * outer
            Jm[:, l, :, m, :] += 0.5 * F[:, l, m][:, None, None] * eye
            Jm[:, l, :, l, :] -= 0.5 * F[:, l, m][:, None, None] * eye
    return Jm.reshape(ne, dp1 * d, dp1 * d)


def oseen_matrix(W, a):
    """N_K(w): u -> 1/2 sum_{m != l} F_{lm}(w) (U_m - U_l), as [ne, (d+1) d, (d+1) d]."""
    ne, dp1, d = W.shape
    F = fluxes(W, a)
    N = np.zeros((ne, dp1, d, dp1, d))
    eye = np.eye(d)
    for l in range(dp1):
        for m in range(dp1):
            if m == l:
                continue
            N[:, l, :, m, :] += 0.5 * F[:, l, m][:, None, None] * eye
            N[:, l, :, l, :] -= 0.5 * F[:, l, m][:, None, None] * eye
    return N.reshape(ne, dp1 * d, dp1 * d)


def gather_local(U_faces, topo):
    """Local face velocities [ne, d+1, d] from global [nf, d]; zero on exterior faces."""
    ef = topo["elem_face"]
    out = U_faces[np.maximum(ef, 0)].copy()
    out[ef < 0] = 0.0
    return out
