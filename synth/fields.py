"""Seeded source terms, element means and linearisation fields.

The method consumes the source only through its element means
f̄_K = (1/|K|) ∫_K f (Section 2, definition of the right-hand side, and
Section 3.1, R_K).  They are computed here once, with a collapsed-coordinate
Gauss-Legendre product rule (Stroud's conical product construction: Duffy's
map of the cube onto the simplex, Gauss-Legendre nodes from numpy), and both
the oracle and the library receive the same f̄_K array.
"""

import math

import numpy as np

from .mesh import mesh2d_square, mesh3d_kuhn, batch_sizes

TWO_PI = 2.0 * math.pi


# ----------------------------------------------------------------------------
# Fourier source: f^(i)(x) = sum_m sin(2 pi k_{i,m} . x + phi_{i,m})
# ----------------------------------------------------------------------------
def fourier_modes(d, seed, m=8, kmax=4):
    """Integer wave vectors k in {1..kmax}^d and phases in [0, 2 pi) per component."""
    rng = np.random.default_rng(seed)
    k = rng.integers(1, kmax + 1, size=(d, m, d)).astype(np.float64)
    phi = rng.uniform(0.0, TWO_PI, size=(d, m))
    return {"k": k, "phi": phi}


def fourier_force(x, modes):
    """Evaluate the Fourier source at points x [..., d]; returns [..., d]."""
    k, phi = modes["k"], modes["phi"]
    d = k.shape[0]
    out = np.empty(x.shape[:-1] + (d,), dtype=np.float64)
    for i in range(d):
        theta = TWO_PI * np.einsum("...j,mj->...m", x, k[i]) + phi[i]
        out[..., i] = np.sin(theta).sum(axis=-1)
    return out


# ----------------------------------------------------------------------------
# Element means by a collapsed Gauss-Legendre product rule
# ----------------------------------------------------------------------------
def _simplex_rule(d, q):
    """Barycentric nodes [P, d+1] and weights [P] (summing to 1) on a d-simplex."""
    t, w = np.polynomial.legendre.leggauss(q)
    t = 0.5 * (t + 1.0)
    w = 0.5 * w
    if d == 2:
        u, v = np.meshgrid(t, t, indexing="ij")
        wu, wv = np.meshgrid(w, w, indexing="ij")
        xi, eta = u, v * (1.0 - u)
        wt = wu * wv * (1.0 - u)
        lam = np.stack([1.0 - xi - eta, xi, eta], axis=-1).reshape(-1, 3)
    elif d == 3:
        u, v, s = np.meshgrid(t, t, t, indexing="ij")
        wu, wv, ws = np.meshgrid(w, w, w, indexing="ij")
        xi = u
        eta = v * (1.0 - u)
        zeta = s * (1.0 - u) * (1.0 - v)
        wt = wu * wv * ws * (1.0 - u) ** 2 * (1.0 - v)
        lam = np.stack([1.0 - xi - eta - zeta, xi, eta, zeta], axis=-1).reshape(-1, 4)
    else:
        raise ValueError("d must be 2 or 3")
    wt = wt.ravel()
    return lam, wt / wt.sum()


def element_means(f, coords, elems, order=3, chunk=1 << 18):
    """f̄_K for every element: the mean of the vector field f over K.

    f maps points [P, d] to values [P, d].  Returns float64 [ne, d].
    """
    d = coords.shape[1]
    lam, wt = _simplex_rule(d, order)
    out = np.empty((elems.shape[0], d), dtype=np.float64)
    for s in range(0, elems.shape[0], chunk):
        X = coords[elems[s:s + chunk]]                      # [c, d+1, d]
        pts = np.einsum("pv,cvd->cpd", lam, X)              # [c, P, d]
        vals = f(pts.reshape(-1, d)).reshape(pts.shape)      # [c, P, d]
        out[s:s + chunk] = np.einsum("p,cpd->cd", wt, vals)
    return out


# ----------------------------------------------------------------------------
# Manufactured transient Stokes solution: u = curl psi, psi = prod sin^2(pi x_i)
# ----------------------------------------------------------------------------
def _s0(t):
    return np.sin(math.pi * t) ** 2


def _s1(t):
    return math.pi * np.sin(TWO_PI * t)


def _s2(t):
    return 2.0 * math.pi ** 2 * np.cos(TWO_PI * t)


def _s3(t):
    return -4.0 * math.pi ** 3 * np.sin(TWO_PI * t)


def manufactured_stokes(d, mu, nu, pressure=False):
    """Exact (u, p, f) of mu u - nu Lap u + grad p = f, div u = 0, u = 0 on the boundary.

    psi = prod_i sin^2(pi x_i); u = (d psi/dy, -d psi/dx [, 0]), which is
    divergence free and vanishes on the boundary of the unit square or cube.
    p = 0, or p = sin(2 pi x) sin(2 pi y) (zero mean) when ``pressure``.
    Returns three callables on points [P, d].
    """

    def parts(x):
        cx, cy = x[:, 0], x[:, 1]
        cz = x[:, 2] if d == 3 else None
        S = [_s0(cx), _s0(cy)]
        S1 = [_s1(cx), _s1(cy)]
        S2 = [_s2(cx), _s2(cy)]
        S3 = [_s3(cx), _s3(cy)]
        if d == 3:
            Z0, Z2 = _s0(cz), _s2(cz)
        else:
            Z0, Z2 = np.ones_like(cx), np.zeros_like(cx)
        return S, S1, S2, S3, Z0, Z2

    def u(x):
        S, S1, _, _, Z0, _ = parts(x)
        out = np.zeros_like(x)
        out[:, 0] = S[0] * S1[1] * Z0
        out[:, 1] = -S1[0] * S[1] * Z0
        return out

    def lap_u(x):
        S, S1, S2, S3, Z0, Z2 = parts(x)
        out = np.zeros_like(x)
        out[:, 0] = S2[0] * S1[1] * Z0 + S[0] * S3[1] * Z0 + S[0] * S1[1] * Z2
        out[:, 1] = -(S3[0] * S[1] * Z0 + S1[0] * S2[1] * Z0 + S1[0] * S[1] * Z2)
        return out

    def p(x):
        if not pressure:
            return np.zeros(x.shape[0])
        return np.sin(TWO_PI * x[:, 0]) * np.sin(TWO_PI * x[:, 1])

    def grad_p(x):
        out = np.zeros_like(x)
        if pressure:
            out[:, 0] = TWO_PI * np.cos(TWO_PI * x[:, 0]) * np.sin(TWO_PI * x[:, 1])
            out[:, 1] = TWO_PI * np.sin(TWO_PI * x[:, 0]) * np.cos(TWO_PI * x[:, 1])
        return out

    def f(x):
        return mu * u(x) - nu * lap_u(x) + grad_p(x)

    return {"u": u, "p": p, "f": f, "lap_u": lap_u}


# ----------------------------------------------------------------------------
# Divergence-free linearisation field for a Navier-Stokes step
# ----------------------------------------------------------------------------
def stream_velocity(points, seed=3, m=8, kmax=4):
    """w = curl psi_w at points [P, d], scaled so that max |w| = 1.

    psi_w = prod_i sin^2(pi x_i) * sum_m sin(2 pi k_m . x + phi_m), with
    k_m in {1..kmax}^d and phi_m in [0, 2 pi) from default_rng(seed);
    w = (d psi/dy, -d psi/dx [, 0]).  The scale is fixed on a 257^2 (2D) or
    65^3 (3D) reference grid, so it does not depend on the points asked for.
    """
    d = points.shape[1]
    rng = np.random.default_rng(seed)
    k = rng.integers(1, kmax + 1, size=(m, d)).astype(np.float64)
    phi = rng.uniform(0.0, TWO_PI, size=m)

    def raw(x):
        g = np.ones(x.shape[0])
        gp = []
        for j in range(d):
            g = g * _s0(x[:, j])
        for j in range(d):
            other = np.ones(x.shape[0])
            for i in range(d):
                if i != j:
                    other = other * _s0(x[:, i])
            gp.append(_s1(x[:, j]) * other)
        theta = TWO_PI * x @ k.T + phi
        h = np.sin(theta).sum(axis=1)
        hp = [(TWO_PI * np.cos(theta) * k[:, j]).sum(axis=1) for j in range(d)]
        dpsi = [gp[j] * h + g * hp[j] for j in range(d)]
        w = np.zeros_like(x)
        w[:, 0] = dpsi[1]
        w[:, 1] = -dpsi[0]
        return w

    r = 257 if d == 2 else 65
    axes = [np.linspace(0.0, 1.0, r)] * d
    grid = np.stack([a.ravel() for a in np.meshgrid(*axes, indexing="ij")], axis=1)
    scale = np.sqrt((raw(grid) ** 2).sum(axis=1)).max()
    return raw(points) / scale


# ----------------------------------------------------------------------------
# The five workloads (sizes can be shrunk for tests)
# ----------------------------------------------------------------------------
def config_problem(name, n=None, nrhs=None, quad_order=None):
    """Mesh, coefficients and element-mean sources of one workload.

    cfg1: 2D 16^2, nu=1, mu=100 (dt=1e-2), manufactured curl source, p = 0.
    cfg2: 2D 512^2 perturbed +-0.2h (seed 0), nu=1, mu=1000, Fourier (seed 1).
    cfg3: 3D 64^3 Kuhn, nu=1, mu=1000, Fourier (seed 1).
    cfg5: 2D 1024^2, nu=0.01, mu=0, Newton step about stream_velocity(seed 3),
          Fourier (seed 1).
    Right-hand side j of a multi-RHS problem uses Fourier seed 1 + 1000 j.
    Returns a dict with keys dim, coords, elems, nu, mu, conv, fbar [nrhs, ne, d].
    """
    if name == "cfg1":
        n = 16 if n is None else n
        coords, elems = mesh2d_square(n)
        nu, mu, conv = 1.0, 100.0, "none"
        ms = manufactured_stokes(2, mu, nu)
        fbar = element_means(ms["f"], coords, elems, order=quad_order or 5)[None]
    elif name in ("cfg2", "cfg5"):
        if name == "cfg2":
            n = 512 if n is None else n
            coords, elems = mesh2d_square(n, perturb=0.2, seed=0)
            nu, mu, conv = 1.0, 1000.0, "none"
        else:
            n = 1024 if n is None else n
            coords, elems = mesh2d_square(n)
            nu, mu, conv = 0.01, 0.0, "newton"
        nr = 1 if nrhs is None else nrhs
        fbar = np.stack([
            element_means(lambda x, md=fourier_modes(2, 1 + 1000 * j): fourier_force(x, md),
                          coords, elems, order=quad_order or 3)
            for j in range(nr)])
    elif name == "cfg3":
        n = 64 if n is None else n
        coords, elems = mesh3d_kuhn(n)
        nu, mu, conv = 1.0, 1000.0, "none"
        nr = 1 if nrhs is None else nrhs
        fbar = np.stack([
            element_means(lambda x, md=fourier_modes(3, 1 + 1000 * j): fourier_force(x, md),
                          coords, elems, order=quad_order or 2)
            for j in range(nr)])
    else:
        raise ValueError(f"unknown workload {name}")
    return {"name": name, "n": n, "dim": coords.shape[1], "coords": coords, "elems": elems,
            "nu": nu, "mu": mu, "conv": conv, "fbar": np.ascontiguousarray(fbar)}


def batch_problems(count=64, nrhs=4, lo=8, hi=256, seed=2, mu=1000.0, nu=1.0):
    """The batched workload: ``count`` perturbed 2D meshes with ``nrhs`` Fourier sources each."""
    probs = []
    for p, n in enumerate(batch_sizes(count, lo, hi, seed)):
        coords, elems = mesh2d_square(n, perturb=0.2, seed=p)
        fbar = np.stack([
            element_means(lambda x, md=fourier_modes(2, 1 + 1000 * j): fourier_force(x, md),
                          coords, elems, order=3)
            for j in range(nrhs)])
        probs.append({"n": n, "dim": 2, "coords": coords, "elems": elems, "nu": nu, "mu": mu,
                      "conv": "none", "fbar": fbar})
    return probs
