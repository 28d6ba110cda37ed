"""Textbook Krylov solvers for G W = S (Section 3.2, hybrid method step 2).

The paper solves the SPD system of transient Stokes by "a simple
preconditioned conjugate gradient" and the nonsymmetric systems of the
Newton steps by GMRES (Section 4.3).  These are the standard algorithms
(Saad, Iterative Methods for Sparse Linear Systems: Algorithm 9.1,
preconditioned CG; Algorithm 9.5, right-preconditioned restarted GMRES with
Givens rotations), written plainly; the preconditioner is Jacobi (the
inverse of the diagonal of G).  ``minres`` is Paige and Saunders' MINRES
with a diagonal preconditioner, for the symmetric indefinite coupled system
of Eq. 10 solved without hybridisation.  ``refine`` is classical mixed-precision
iterative refinement: inner solves in float32, residual and update in float64.
``chebyshev_pcg`` is CG with a polynomial preconditioner (a fixed number of
Jacobi-preconditioned Chebyshev steps, Saad Algorithm 12.1) on the interval
below a Gershgorin bound of the spectrum.  ``deflated_pcg`` keeps the CG
directions G-orthogonal to given vectors (deflated CG), removing their
eigenvalues from the convergence; ``lanczos_ritz`` takes approximate low
eigenvectors of the preconditioned operator from the coefficients and
preconditioned residuals of a PCG run (the Lanczos connection of CG), the
vectors a later solve with the same G deflates.
"""

import numpy as np


def jacobi(G):
    """Inverse of the diagonal of G."""
    return 1.0 / G.diagonal()


def pcg(G, b, minv, x0=None, rtol=1e-10, maxit=100000):
    """Jacobi-preconditioned CG; stops when ||r||_2 <= rtol ||b||_2 (recursive r)."""
    dt = b.dtype
    x = np.zeros_like(b) if x0 is None else x0.astype(dt).copy()
    r = b - G @ x
    bn = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / bn if bn > 0 else 0.0]
    if bn == 0.0:
        return x, 0, hist
    z = minv * r
    p = z.copy()
    rz = np.dot(r, z)
    it = 0
    while it < maxit:
        q = G @ p
        alpha = rz / np.dot(p, q)
        x += alpha * p
        r -= alpha * q
        it += 1
        rn = np.linalg.norm(r) / bn
        hist.append(rn)
        if rn <= rtol:
            break
        z = minv * r
        rz_new = np.dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, hist


def gershgorin_bound(G, minv):
    """Upper bound of the eigenvalues of M^{-1} G, M^{-1} = diag(minv) > 0:
    the largest absolute row sum of M^{-1} G (Gershgorin's circle theorem)."""
    rows = np.asarray(abs(G).sum(axis=1)).ravel()
    return float(np.max(rows * np.abs(minv)))


def chebyshev_apply(G, minv, r, degree, lmax, ratio):
    """Polynomial preconditioner z = P(r) for SPD G: `degree` steps of the
    Chebyshev iteration on G z = r, Jacobi-preconditioned by diag(minv), from
    z = 0, for the interval [lmax/ratio, lmax] (Saad, Iterative Methods for
    Sparse Linear Systems, Algorithm 12.1, applied to M^{-1} G z = M^{-1} r).

    With theta, delta the centre and half width of the interval and
    sigma = theta/delta: d_0 = M^{-1} r / theta, rho_0 = 1/sigma, and for
    j = 0 .. degree-1: z_{j+1} = z_j + d_j; then (if another step follows)
    res = r - G z_{j+1}, rho_{j+1} = 1/(2 sigma - rho_j),
    d_{j+1} = rho_{j+1} rho_j d_j + (2 rho_{j+1}/delta) M^{-1} res.
    On an eigenvector v of M^{-1} G with eigenvalue lam, M^{-1} r = v gives
    z = (1 - T_k((theta - lam)/delta) / T_k(sigma)) / lam * v (T_k the
    Chebyshev polynomial, k = degree): positive for 0 < lam <= lmax, so P is
    symmetric positive definite when lmax bounds the spectrum.  degree - 1
    products with G."""
    a, b = lmax / ratio, lmax
    theta, delta = 0.5 * (b + a), 0.5 * (b - a)
    sigma = theta / delta
    rho = 1.0 / sigma
    d = minv * r / theta
    z = np.zeros_like(r)
    for j in range(degree):
        z = z + d
        if j == degree - 1:
            break
        res = r - G @ z
        rho_next = 1.0 / (2.0 * sigma - rho)
        d = rho_next * rho * d + (2.0 * rho_next / delta) * (minv * res)
        rho = rho_next
    return z


def chebyshev_pcg(G, b, minv, degree, ratio, lmax=None, x0=None, rtol=1e-10, maxit=100000):
    """CG preconditioned by chebyshev_apply (Saad, Algorithm 9.1 with the
    polynomial preconditioner); lmax defaults to gershgorin_bound(G, minv).
    Stops when ||r||_2 <= rtol ||b||_2 (recursive r).  Returns (x, iterations,
    history of ||r||/||b||); each iteration applies G `degree` times."""
    if lmax is None:
        lmax = gershgorin_bound(G, minv)
    x = np.zeros_like(b) if x0 is None else x0.astype(b.dtype).copy()
    r = b - G @ x
    bn = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / bn if bn > 0 else 0.0]
    if bn == 0.0:
        return x, 0, hist
    z = chebyshev_apply(G, minv, r, degree, lmax, ratio)
    p = z.copy()
    rz = np.dot(r, z)
    it = 0
    while it < maxit:
        q = G @ p
        alpha = rz / np.dot(p, q)
        x += alpha * p
        r -= alpha * q
        it += 1
        rn = np.linalg.norm(r) / bn
        hist.append(rn)
        if rn <= rtol:
            break
        z = chebyshev_apply(G, minv, r, degree, lmax, ratio)
        rz_new = np.dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, hist


def deflated_pcg(G, b, precond, V, rtol=1e-10, maxit=100000):
    """CG on G x = b with the directions kept G-orthogonal to the columns of V
    (deflated CG: Saad, Yeung, Erhel and Guyomarc'h, SIAM J. Sci. Comput. 21,
    2000), preconditioned by the function `precond` (z = precond(r)).

    With E = V^t G V: x_0 = V E^{-1} V^t b, so that V^t r_0 = 0; then
    z = precond(r), p = z + beta p - V E^{-1} (G V)^t z.  Every residual stays
    orthogonal to V, and the eigenvalues of the columns of V drop out of the
    convergence.  V may have no columns (plain PCG).  Stops when
    ||r||_2 <= rtol ||b||_2 (recursive r).  Returns (x, iterations, history)."""
    V = np.asarray(V, dtype=b.dtype).reshape(b.shape[0], -1)
    GV = G @ V if V.shape[1] else V
    E = V.T @ GV

    def project(z):   # remove the G-components along V
        return z - V @ np.linalg.solve(E, GV.T @ z) if V.shape[1] else z

    x = V @ np.linalg.solve(E, V.T @ b) if V.shape[1] else np.zeros_like(b)
    r = b - G @ x
    bn = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / bn if bn > 0 else 0.0]
    if bn == 0.0:
        return x, 0, hist
    z = precond(r)
    p = project(z)
    rz = np.dot(r, z)
    it = 0
    while it < maxit:
        q = G @ p
        alpha = rz / np.dot(p, q)
        x += alpha * p
        r -= alpha * q
        it += 1
        rn = np.linalg.norm(r) / bn
        hist.append(rn)
        if rn <= rtol:
            break
        z = precond(r)
        rz_new = np.dot(r, z)
        p = project(z) + (rz_new / rz) * p
        rz = rz_new
    return x, it, hist


def lanczos_ritz(G, b, precond, m, k):
    """Ritz pairs of the preconditioned operator from m steps of PCG on G x = b
    from x = 0 (Saad, Iterative Methods for Sparse Linear Systems, Section 6.7.3,
    the Lanczos connection of CG), preconditioner z = precond(r) with M its inverse.

    The preconditioned residuals z_j of PCG satisfy z_i . r_j = 0 for i != j, so
    q_j = z_j / sqrt(r_j . z_j) are orthonormal in the inner product of M, and
    Q^t G Q (Q = [q_0 .. q_{m-1}]) is the tridiagonal matrix T whose entries
    follow from the CG step lengths alpha_j and the ratios beta_j = r_{j+1}.z_{j+1}
    / r_j.z_j:
        T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}   (no second term for j = 0),
        T_{j,j+1} = T_{j+1,j} = -sqrt(beta_j)/alpha_j.
    The eigenpairs (theta, s) of T with the k smallest theta give the Ritz
    vectors y = Q s, approximate eigenvectors of M^{-1} G (Galerkin condition:
    Q^t (G y - theta M y) = 0).  Stops early when the
    residual vanishes.  Returns (theta [k'], Y [n, k'], T [m', m']) with m' the
    steps taken and k' = min(k, m')."""
    r = np.array(b, dtype=float, copy=True)
    z = precond(r)
    rz = float(np.dot(r, z))
    p = z.copy()
    Q, alphas, betas = [], [], []
    for _ in range(m):
        if not rz > 0.0:
            break
        Q.append(z / np.sqrt(rz))
        q = G @ p
        alpha = rz / float(np.dot(p, q))
        alphas.append(alpha)
        r = r - alpha * q
        z = precond(r)
        rz_new = float(np.dot(r, z))
        beta = rz_new / rz
        betas.append(beta)
        p = z + beta * p
        rz = rz_new
    mm = len(alphas)
    T = np.zeros((mm, mm))
    for j in range(mm):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < mm:
            T[j, j + 1] = T[j + 1, j] = -np.sqrt(betas[j]) / alphas[j]
    theta, S = np.linalg.eigh(T)
    kk = min(k, mm)
    Qm = np.array(Q).T if mm else np.zeros((b.shape[0], 0))
    return theta[:kk], Qm @ S[:, :kk], T


def gmres(G, b, minv, x0=None, restart=30, rtol=1e-10, maxit=100000):
    """Right-Jacobi-preconditioned restarted GMRES(m) with modified Gram-Schmidt."""
    dt = b.dtype
    n = b.shape[0]
    x = np.zeros_like(b) if x0 is None else x0.astype(dt).copy()
    bn = np.linalg.norm(b)
    hist = []
    if bn == 0.0:
        return x, 0, [0.0]
    it = 0
    while it < maxit:
        r = b - G @ x
        beta = np.linalg.norm(r)
        hist.append(beta / bn)
        if beta / bn <= rtol:
            break
        V = np.zeros((restart + 1, n), dtype=dt)
        H = np.zeros((restart + 1, restart), dtype=np.float64)
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(restart):
            w = G @ (minv * V[j])
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
            hist.append(abs(g[j + 1]) / bn)
            if abs(g[j + 1]) / bn <= rtol or it >= maxit:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        x = x + (minv * (V[:k].T @ y.astype(dt))).astype(dt)
        if hist[-1] <= rtol:
            r = b - G @ x
            if np.linalg.norm(r) / bn <= rtol:
                hist.append(np.linalg.norm(r) / bn)
                break
    return x, it, hist


def minres(K, b, minv, x0=None, rtol=1e-10, maxit=100000):
    """Preconditioned MINRES (Paige and Saunders) for a symmetric, possibly
    indefinite K with a symmetric positive semidefinite diagonal preconditioner
    minv (entries 0 remove their unknown from the Krylov space).

    The Lanczos process runs in the M-inner product (M^{-1} = diag(minv)):
    v_1 = r_0, z_j = M^{-1} v_j, gamma_j = sqrt(z_j . v_j); the tridiagonal
    system is reduced by Givens rotations (c, s) and the iterate is updated
    along directions w_j, so that |eta| = ||b - K x_j||_{M^{-1}} after step j.
    Stops when |eta| <= rtol * gamma_1, or after maxit steps.  Returns
    (x, steps, history of |eta| / gamma_1).
    """
    x = np.zeros_like(b) if x0 is None else x0.astype(b.dtype).copy()
    v_old = np.zeros_like(b)
    v = b - K @ x
    z = minv * v
    gamma = np.sqrt(np.dot(z, v))
    gamma1 = gamma
    hist = [1.0 if gamma1 > 0 else 0.0]
    if gamma1 == 0.0:
        return x, 0, hist
    gamma_old = 1.0
    eta = gamma
    c_old, c = 1.0, 1.0
    s_old, s = 0.0, 0.0
    w_old = np.zeros_like(b)
    w = np.zeros_like(b)
    it = 0
    while it < maxit:
        z = z / gamma
        q = K @ z
        delta = np.dot(q, z)
        v_new = q - (delta / gamma) * v - (gamma / gamma_old) * v_old
        z_new = minv * v_new
        gamma_new = np.sqrt(max(np.dot(z_new, v_new), 0.0))
        # the new column of the tridiagonal matrix, rotated by the last two rotations
        a0 = c * delta - c_old * s * gamma
        a1 = np.hypot(a0, gamma_new)
        a2 = s * delta + c_old * c * gamma
        a3 = s_old * gamma
        c_old, s_old = c, s
        c, s = a0 / a1, gamma_new / a1
        w_new = (z - a3 * w_old - a2 * w) / a1
        x = x + c * eta * w_new
        eta = -s * eta
        it += 1
        hist.append(abs(eta) / gamma1)
        if abs(eta) <= rtol * gamma1 or gamma_new == 0.0:
            break
        v_old, v = v, v_new
        z = z_new
        gamma_old, gamma = gamma, gamma_new
        w_old, w = w, w_new
    return x, it, hist


def refine(G, b, inner="pcg", rtol=1e-10, inner_rtol=1e-4, max_outer=60, restart=30,
           inner_maxit=100000):
    """float64 iterative refinement around a float32 inner Krylov solve.

    x = 0; repeat: r = b - G x (float64); solve G d = r in float32 to a
    relative residual inner_rtol; x += d (float64); until ||r|| <= rtol ||b||.
    Returns (x, outer steps, total inner iterations, history of ||r||/||b||).
    """
    G32 = G.astype(np.float32)
    minv32 = jacobi(G).astype(np.float32)
    x = np.zeros_like(b)
    bn = np.linalg.norm(b)
    hist = []
    inner_total = 0
    outer = 0
    while True:
        r = b - G @ x
        rn = np.linalg.norm(r) / bn if bn > 0 else 0.0
        hist.append(rn)
        if rn <= rtol or outer >= max_outer:
            break
        r32 = r.astype(np.float32)
        if inner == "pcg":
            dx, k, _ = pcg(G32, r32, minv32, rtol=inner_rtol, maxit=inner_maxit)
        else:
            dx, k, _ = gmres(G32, r32, minv32, restart=restart, rtol=inner_rtol, maxit=inner_maxit)
        x += dx.astype(np.float64)
        inner_total += k
        outer += 1
    return x, outer, inner_total, hist
