"""End-to-end oracle runs: the coupled direct solve and the hybrid method.

``direct`` is the plain definition (Eq. 10 solved by a library direct
solver); ``hybrid`` follows the three steps of the hybrid method
(Section 3.2, closing list): compute G and S, solve G W = S, recover P and U.
"""

import time

import numpy as np
import scipy.sparse.linalg as spla

from . import coupled, elements, hybrid as hyb_mod, krylov, topology


def setup(coords, elems, nu, mu, fbar, conv="none", w=None, u_prev=None):
    """Topology, geometry and element blocks (Sections 2 and 3.1); u_prev: the
    previous level of an implicit Euler step, or None."""
    topo = topology.build_faces(elems)
    geom = elements.geometry(coords, elems)
    A_K, D_K, R_K = coupled.element_blocks(topo, geom, nu, mu, fbar, conv, w, u_prev)
    return topo, geom, A_K, D_K, R_K


def face_centroids(coords, topo):
    """Centroid x_sigma of each interior face, in the oracle's face order."""
    return np.asarray(coords)[topo["face_vertices"]].mean(axis=1)


def direct(coords, elems, nu, mu, fbar, conv="none", w=None, k0=0, dense=False, u_prev=None):
    """U [nf, d] and P [ne] (P_{K_0} = 0) of Eq. 10 by a direct solve."""
    topo, geom, A_K, D_K, R_K = setup(coords, elems, nu, mu, fbar, conv, w, u_prev)
    A, D, R = coupled.assemble(topo, A_K, D_K, R_K, k0)
    U, P = coupled.solve_direct(A, D, R, k0, dense=dense)
    return {"U": U.reshape(-1, topo["d"]), "P": P, "topo": topo, "geom": geom,
            "A": A, "D": D, "R": R}


def hybrid(coords, elems, nu, mu, fbar, conv="none", w=None, k0=0, method="direct",
           rtol=1e-12, inner_rtol=1e-4, restart=30, lam_scale=2.0, maxit=100000):
    """The hybrid method; method in {direct, pcg, gmres, ir-pcg, ir-gmres}."""
    t0 = time.perf_counter()
    topo, geom, A_K, D_K, R_K = setup(coords, elems, nu, mu, fbar, conv, w)
    h = hyb_mod.hybridise(topo, A_K, D_K, R_K, mu, k0, lam_scale)
    t1 = time.perf_counter()
    G, S = h["G"], h["S"]
    stats = {"method": method}
    if S.size == 0 or not np.any(S):
        W = np.zeros_like(S)
        stats["iters"] = 0
    elif method == "direct":
        W = spla.spsolve(G.tocsc(), S)
        stats["iters"] = 0
    elif method == "pcg":
        W, it, hist = krylov.pcg(G, S, krylov.jacobi(G), rtol=rtol, maxit=maxit)
        stats.update(iters=it, hist=hist)
    elif method == "gmres":
        W, it, hist = krylov.gmres(G, S, krylov.jacobi(G), restart=restart, rtol=rtol, maxit=maxit)
        stats.update(iters=it, hist=hist)
    elif method in ("ir-pcg", "ir-gmres"):
        W, outer, inner, hist = krylov.refine(G, S, inner=method[3:], rtol=rtol,
                                              inner_rtol=inner_rtol, restart=restart)
        stats.update(iters=inner, outer=outer, hist=hist)
    else:
        raise ValueError(method)
    t2 = time.perf_counter()
    U, P, jump = hyb_mod.recover(h, topo, W)
    t3 = time.perf_counter()
    stats.update(t_hybridise=t1 - t0, t_solve=t2 - t1, t_recover=t3 - t2, jump=jump)
    if S.size:
        stats["relres"] = float(np.linalg.norm(S - G @ W) / max(np.linalg.norm(S), 1e-300))
    return {"U": U.reshape(-1, topo["d"]), "P": P, "W": W.reshape(-1, topo["d"]),
            "topo": topo, "geom": geom, "hyb": h, "stats": stats,
            "A_K": A_K, "D_K": D_K, "R_K": R_K}
