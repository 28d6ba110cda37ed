"""The coupled velocity-pressure system of Eq. 10 and its direct solve.

This is the plain definition of the result the hybrid method reaches
exactly (Section 3.2, item 2): assemble A = sum_K H_K A_K H_K^t,
D = sum_{K != K_0} F_K D_K^t H_K^t, R = sum_K H_K R_K (Section 3.1) and
solve [A D^t; D 0][U; P] = [R; 0] with a library direct solver.
Global velocity unknowns are ordered face*d + i; pressures P_K for
K != K_0 in increasing simplex order.
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import convection, elements, krylov


def element_blocks(topo, geom, nu, mu, fbar, conv="none", w=None, u_prev=None):
    """A_K, D_K, R_K for every simplex, zero outside the interior unknowns.

    conv = "none": A_K = S_K (x) Id (Section 3.1).
    conv = "newton": A_K is completed with the derivative of the convection
      term at w and R_K with the Newton term; since b_h is quadratic the
      linear system (S + J(w)) u + D^t P = R - c(w) + J(w) w reads
      (S + J(w)) u + D^t P = R + c(w)  (Section 3.1, b_h != 0).
    conv = "oseen": A_K += N_K(w), R_K unchanged (Picard linearisation).
    fbar [ne, d]; w [nf, d] face velocities about which to linearise.
    u_prev [nf, d] or None: the previous time level of an implicit Euler step
      (mu = 1/dt), whose lumped mass term joins R_K (elements.local_R_previous).
    """
    S = elements.local_S(geom, nu, mu)
    A = elements.local_A(S)
    D = elements.local_D(geom)
    R = elements.local_R(geom, fbar)
    if u_prev is not None:
        R = R + elements.local_R_previous(topo, geom, mu, u_prev)
    if conv != "none":
        Wl = convection.gather_local(np.asarray(w, dtype=np.float64), topo)
        if conv == "newton":
            A = A + convection.newton_jacobian(Wl, geom["a"])
            R = R + convection.element_convection(Wl, geom["a"]).reshape(R.shape)
        elif conv == "oseen":
            A = A + convection.oseen_matrix(Wl, geom["a"])
        else:
            raise ValueError(conv)
    m = elements.interior_mask(topo).astype(np.float64)
    return A * m[:, :, None] * m[:, None, :], D * m, R * m


def assemble(topo, A_K, D_K, R_K, k0=0):
    """Global A (CSR), D (CSR) and R of Eq. 10 from the element blocks."""
    d, ne, nf = topo["d"], topo["ne"], topo["nf"]
    N = nf * d
    dofs = elements.local_dofs(topo)
    nl = dofs.shape[1]
    rows = np.repeat(dofs, nl, axis=1).ravel()
    cols = np.tile(dofs, (1, nl)).ravel()
    vals = A_K.reshape(ne, -1).ravel()
    keep = (rows >= 0) & (cols >= 0)
    A = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(N, N)).tocsr()
    prow = np.arange(ne) - (np.arange(ne) > k0)
    erow = np.repeat(prow[:, None], nl, axis=1)
    keepd = (dofs >= 0) & (np.arange(ne) != k0)[:, None]
    D = sp.coo_matrix((D_K[keepd], (erow[keepd], dofs[keepd])), shape=(ne - 1, N)).tocsr()
    R = np.zeros(N)
    keepr = dofs >= 0
    np.add.at(R, dofs[keepr], R_K[keepr])
    return A, D, R


def saddle_matrix(A, D):
    """[A D^t; D 0] as CSR."""
    return sp.bmat([[A, D.T], [D, None]], format="csr")


def saddle_preconditioner(A, D):
    """Diagonal preconditioner of [A D^t; D 0] for MINRES: 1/diag(A) on the
    velocities and 1/diag(D diag(A)^{-1} D^t) on the pressures (the diagonal
    of the Schur complement with A replaced by its diagonal)."""
    da = A.diagonal()
    schur = np.asarray((D.multiply(D)) @ (1.0 / da)).ravel()
    return np.concatenate([1.0 / da, 1.0 / schur])


def solve_minres(A, D, R, rtol=1e-10, maxit=1000000, k0=0):
    """Eq. 10 without hybridisation: preconditioned MINRES on the coupled
    system (the comparison the paper draws against the hybrid method);
    returns U, P (P_{K_0} = 0), the MINRES steps and the history."""
    N = A.shape[0]
    ne = D.shape[0] + 1
    K = saddle_matrix(A, D)
    rhs = np.concatenate([R, np.zeros(ne - 1)])
    sol, it, hist = krylov.minres(K, rhs, saddle_preconditioner(A, D), rtol=rtol, maxit=maxit)
    return sol[:N], np.insert(sol[N:], k0, 0.0), it, hist


def solve_direct(A, D, R, k0=0, dense=False):
    """Direct solve of Eq. 10; returns U [nf, d]-flattened and P [ne] with P_{K_0} = 0."""
    N = A.shape[0]
    ne = D.shape[0] + 1
    M = saddle_matrix(A, D)
    rhs = np.concatenate([R, np.zeros(ne - 1)])
    if dense:
        sol = np.linalg.solve(M.toarray(), rhs)
    else:
        sol = spla.spsolve(M.tocsc(), rhs)
    U = sol[:N]
    P = np.insert(sol[N:], k0, 0.0)
    return U, P


def coupled_residual(A, D, R, U, P, k0=0):
    """|| [A D^t; D 0][U; P] - [R; 0] ||_2 / ||R||_2 for a candidate solution."""
    Pr = np.delete(P, k0)
    r1 = A @ U + D.T @ Pr - R
    r2 = D @ U
    return float(np.sqrt(np.dot(r1, r1) + np.dot(r2, r2)) / max(np.linalg.norm(R), 1e-300))


def normalise_pressure(P, vol):
    """P - (1/|Omega|) int_Omega P: the zero-mean representative (Section 2, item 5)."""
    return P - np.dot(vol, P) / vol.sum()
