"""Steady problems (mu = 0) solved with transient hybridised solves as preconditioner.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The steady coupled system of Eq. 10 with mu = 0,
    K_s [U; P] = [R; 0],   K_s = [A_0 D^t; D 0],   P_{K_0} = 0,
is what the hybrid method with the E_K stabilisation of Section 3.2 (item 7)
eliminates to an indefinite G.  Here it is solved by flexible GMRES (Saad,
Iterative Methods for Sparse Linear Systems, Algorithm 9.6) on K_s itself,
right-preconditioned by the transient coupled operator
    K_mu = [A_0 + mu M, D^t; D 0]
(the same problem with the lumped mass M of S_K added, Section 3.1), which
the hybrid method solves exactly with an SPD G when the convection term is
absent (Section 3.2, item 6).  A residual [v; g] enters K_mu^{-1} as follows:
v is the right-hand side of an implicit Euler step from the previous level
u_prev = v / (mu m) with zero source, m_sigma = sum_{K ni sigma} |K|/(d+1)
(elements.local_R_previous assembles mu m u_prev = v); g is a non-zero
divergence D_K^t U_K = g_K per simplex, which the element-wise elimination of
Section 3.2 (items 2-4) carries through: P_K = (D_K^t Â^{-1} y - g_K)/B_K, so
Û_K = M_K y + Â^{-1} D_K g_K / B_K and S gains sum_K H_K C_K Â^{-1} D_K g_K / B_K
(g_{K_0} plays no part: P_{K_0} = 0).  On divergence-free velocities K_s
K_mu^{-1} has the eigenvalues lambda/(lambda + mu), lambda those of the steady
operator, so the number of outer steps does not depend on the mesh.  The
flexible form keeps the minimised residual that of K_s whatever the inner
solves return; with the divergence block carried, inner solves to 1e-4 do.
"""

import numpy as np
import scipy.sparse.linalg as spla

from . import coupled, elements, hybrid, pipeline


def face_mass(topo, geom):
    """m_sigma = sum over the simplices K of sigma of |K|/(d+1), per interior face [nf]."""
    d = topo["d"]
    m = np.zeros(topo["nf"])
    ef = topo["elem_face"]
    share = geom["vol"] / (d + 1)
    for l in range(d + 1):
        inside = ef[:, l] >= 0
        np.add.at(m, ef[inside, l], share[inside])
    return m


class TransientPreconditioner:
    """z = K_mu^{-1} [v; 0] by the hybrid method on the transient system (nu, mu,
    conv, w) of the mesh: G_mu W = S(v), then the element-wise recovery.
    solve(G, S) solves the hybridised system (default: a sparse LU of G_mu)."""

    def __init__(self, coords, elems, nu, mu, conv="none", w=None, solve=None):
        if not mu > 0.0:
            raise ValueError("the preconditioning transient system needs mu > 0")
        self.mu = mu
        self.d = coords.shape[1]
        ne = elems.shape[0]
        zero = np.zeros((ne, self.d))
        self.topo, self.geom, A_K, self.D_K, _ = pipeline.setup(coords, elems, nu, mu, zero, conv, w)
        self.A_K = A_K
        self.h = hybrid.hybridise(self.topo, A_K, self.D_K, np.zeros((ne, A_K.shape[1])), mu)
        self.m = np.repeat(face_mass(self.topo, self.geom), self.d)
        if solve is None:
            lu = spla.splu(self.h["G"].tocsc())
            solve = lambda G, S: lu.solve(S)   # noqa: E731
        self.solve = solve
        self.applications = 0

    def __call__(self, v, g=None):
        """(z_u [N], z_p [ne] with z_p[K_0] = 0) solving K_mu [z_u; z_p] = [v; g] for
        the velocity residual v [N] and the divergence residual g [ne] (None: 0;
        the entry of K_0 is not used)."""
        u_prev = v / (self.mu * self.m)
        R_K = elements.local_R_previous(self.topo, self.geom, self.mu, u_prev)
        R_K = R_K * elements.interior_mask(self.topo)
        h = self.h
        dofs, Cv, Ainv, D_K, B = h["dofs"], h["Cv"], h["Ainv"], h["D_K"], h["B"]
        k0 = h["k0"]
        gK = np.zeros(B.shape[0]) if g is None else np.asarray(g, dtype=np.float64).copy()
        gK[k0] = 0.0
        invB = 1.0 / np.where(B == 0.0, 1.0, B)
        invB[k0] = 0.0
        u = np.einsum("kab,kb->ka", Ainv, D_K)                       # Â^{-1} D_K
        # S = sum_K H_K C_K (M_K R_K + Â^{-1} D_K g_K / B_K); M_K from G_K = C_K M_K C_K (C_K^2 = 1)
        M = h["GK"] * Cv[:, :, None] * Cv[:, None, :]
        SK = Cv * (np.einsum("kab,kb->ka", M, R_K) + u * (gK * invB)[:, None])
        S = np.zeros(self.m.shape[0])
        kp = dofs >= 0
        np.add.at(S, dofs[kp], SK[kp])
        W = self.solve(self.h["G"], S)
        # recovery (Section 3.2, items 2 and 4) with the divergence g_K
        Wl = np.where(kp, W[np.maximum(dofs, 0)], 0.0)
        y = R_K - Cv * Wl
        Ay = np.einsum("kab,kb->ka", Ainv, y)
        P = (np.einsum("ka,ka->k", D_K, Ay) - gK) * invB
        Uh = Ay - u * P[:, None]
        fe, fl = self.topo["face_elems"], self.topo["face_local"]
        U = Uh.reshape(-1, self.d + 1, self.d)[fe[:, 0], fl[:, 0]].ravel()
        self.applications += 1
        return U, P


def fgmres(apply_K, precond, b, restart=30, rtol=1e-10, maxit=1000):
    """Flexible GMRES(m) (Saad, Algorithm 9.6) with modified Gram-Schmidt.

    apply_K(x) = K x; precond(v) returns z_j for the Arnoldi vector v_j (it may
    change from step to step).  x = x_0 + Z_m y_m, y_m minimising
    ||beta e_1 - H_m y||.  Stops when the residual estimate |g_{j+1}| falls to
    rtol ||b|| and the true residual of the cycle's iterate confirms it.
    Returns (x, steps, history of ||b - K x||/||b||, estimates per step)."""
    n = b.shape[0]
    x = np.zeros(n)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0, [0.0]
    hist = []
    it = 0
    while it < maxit:
        r = b - apply_K(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bn)
        if beta / bn <= rtol:
            break
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(restart):
            Z[j] = precond(V[j])
            w = apply_K(Z[j])
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            it += 1
            if abs(g[j + 1]) / bn <= rtol or it >= maxit:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        x = x + Z[:k].T @ y
    return x, it, hist


def solve_steady(coords, elems, nu, fbar, conv="none", w=None, mu_pre=100.0, pre_conv=None, k0=0,
                 restart=30, rtol=1e-10, maxit=1000, inner=None):
    """U [nf d] and P [ne] (P_{K_0} = 0) of the steady problem (Eq. 10, mu = 0) by
    flexible GMRES on the coupled system, preconditioned by transient hybridised
    solves with mu_pre (conv of the preconditioner: pre_conv, default the
    problem's).  inner(G, S): the hybridised solve (default sparse LU).
    Returns (U, P, stats)."""
    topo, geom, A_K, D_K, R_K = pipeline.setup(coords, elems, nu, 0.0, fbar, conv, w)
    A, D, R = coupled.assemble(topo, A_K, D_K, R_K, k0)
    N, ne = A.shape[0], elems.shape[0]
    pre = TransientPreconditioner(coords, elems, nu, mu_pre, conv if pre_conv is None else pre_conv, w, inner)
    if k0 != 0:
        raise ValueError("the transient preconditioner fixes P at K_0 = 0")

    def apply_K(x):
        u, p = x[:N], x[N:]
        return np.concatenate([A @ u + D.T @ p, D @ u])

    def precond(v):
        zu, zp = pre(v[:N], np.insert(v[N:], k0, 0.0))
        return np.concatenate([zu, zp[1:]])

    b = np.concatenate([R, np.zeros(ne - 1)])
    x, steps, hist = fgmres(apply_K, precond, b, restart=restart, rtol=rtol, maxit=maxit)
    U, P = x[:N], np.insert(x[N:], k0, 0.0)
    return U, P, {"steps": steps, "hist": hist, "applications": pre.applications,
                  "relres": coupled.coupled_residual(A, D, R, U, P, k0)}


def newton(coords, elems, nu, fbar, tol=5e-7, maxit=30):
    """Newton's method for the steady Navier-Stokes problem (Section 3.1 with the
    convection form b_h of Eq. 9, mu = 0): from U_0 = 0, U_{k+1} solves the
    coupled system linearised about w = U_k (coupled.element_blocks with
    conv = "newton": Jacobian of b_h at w, right-hand side R + c(w)) by the
    direct solve; stop when ||U_{k+1} - U_k|| <= tol ||U_{k+1}||.
    Returns (U, P with P_{K_0} = 0, increments per step)."""
    d = coords.shape[1]
    U = np.zeros(0)
    hist = []
    for _ in range(maxit):
        w = U.reshape(-1, d) if U.size else None
        if w is None:
            ref = pipeline.direct(coords, elems, nu, 0.0, fbar)          # w = 0: the Stokes problem
        else:
            ref = pipeline.direct(coords, elems, nu, 0.0, fbar, "newton", w)
        Un = ref["U"].ravel()
        inc = np.linalg.norm(Un - (U if U.size else 0.0)) / np.linalg.norm(Un)
        U, P = Un, ref["P"]
        hist.append(inc)
        if inc <= tol:
            break
    return U, P, hist


def navier_stokes_residual(coords, elems, nu, fbar, U, P, k0=0):
    """||S U + B(U) + D^t P - R|| / ||R|| and ||D U|| / ||R|| for the steady problem,
    B(U) assembled from the element convection terms c_K(U) of Eq. 9."""
    from . import convection
    d = coords.shape[1]
    topo, geom, A_K, D_K, R_K = pipeline.setup(coords, elems, nu, 0.0, fbar)
    A, D, R = coupled.assemble(topo, A_K, D_K, R_K, k0)
    c = convection.element_convection(convection.gather_local(U.reshape(-1, d), topo), geom["a"])
    c = c.reshape(c.shape[0], -1) * elements.interior_mask(topo)
    B = np.zeros_like(R)
    dofs = elements.local_dofs(topo)
    kp = dofs >= 0
    np.add.at(B, dofs[kp], c[kp])
    mom = A @ U + B + D.T @ np.delete(P, k0) - R
    return float(np.linalg.norm(mom) / np.linalg.norm(R)), float(np.linalg.norm(D @ U) / np.linalg.norm(R))
