"""Planted mistakes in the oracle must be caught by its pins.

Each case patches one plausible error into the oracle (on the CPU) and runs
the pin that should catch it; the pin has to fail.
"""

import warnings

import numpy as np
import pytest

from oracle import elements, hybrid, krylov, steady, topology
import test_oracle_chebyshev as tc
import test_oracle_deflation as tdf
import test_oracle_geometry as tg
import test_oracle_krylov as tk
import test_oracle_hybrid as th
import test_oracle_minres as tm
import test_oracle_steady as ts
import test_oracle_time as tt


def wrong_D(geom):
    return geom["a"].reshape(geom["a"].shape[0], -1)           # sign dropped


def wrong_S(geom, nu, mu):
    g = elements.cr_gradients(geom)
    return nu * geom["vol"][:, None, None] * np.einsum("kad,kbd->kab", g, g)   # mass term dropped


def wrong_R(geom, fbar):
    a, xs = geom["a"], geom["xs"]
    rho = np.einsum("kd,kld->kl", fbar, xs)                    # x_K dropped
    return (a * rho[:, :, None]).reshape(a.shape[0], -1)


def wrong_signs(topo):
    return np.abs(topology.__dict__["_orig_owner_signs"](topo))   # C_K + C_L != 0


def wrong_geometry_normal(coords, elems):
    g = topology.__dict__["_orig_geometry"](coords, elems)
    g["a"] = g["a"][:, ::-1]                                    # faces mislabelled
    return g


def wrong_previous(topo, geom, mu, u_prev):
    d = topo["d"]
    ef = topo["elem_face"]
    U = np.asarray(u_prev, dtype=np.float64).reshape(-1, d)
    loc = np.where((ef >= 0)[:, :, None], U[np.maximum(ef, 0)], 0.0)
    return ((mu * geom["vol"] / d)[:, None, None] * loc).reshape(ef.shape[0], -1)   # |K|/d, not |K|/(d+1)


_orig_minres = krylov.minres
_orig_gmres = krylov.gmres


def wrong_gmres(G, b, minv, x0=None, restart=30, rtol=1e-10, maxit=100000):
    # the preconditioner applied twice: another Krylov space
    return _orig_gmres(G, b, minv * minv, x0=x0, restart=restart, rtol=rtol, maxit=maxit)


def wrong_minres(K, b, minv, x0=None, rtol=1e-10, maxit=100000):
    # the preconditioner applied twice: a different (still symmetric) method
    return _orig_minres(K, b, minv * minv, x0=x0, rtol=rtol, maxit=maxit)


def wrong_pcg(G, b, minv, x0=None, rtol=1e-10, maxit=100000):
    # beta from the unpreconditioned residuals (r.r) instead of r.M^{-1}r
    x = np.zeros_like(b) if x0 is None else x0.astype(b.dtype).copy()
    r = b - G @ x
    bn = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / bn]
    z = minv * r
    p = z.copy()
    rz = np.dot(r, z)
    rr = np.dot(r, r)
    it = 0
    while it < maxit:
        q = G @ p
        alpha = rz / np.dot(p, q)
        x += alpha * p
        r -= alpha * q
        it += 1
        hist.append(np.linalg.norm(r) / bn)
        if hist[-1] <= rtol:
            break
        z = minv * r
        rr_new = np.dot(r, r)
        p = z + (rr_new / rr) * p
        rz, rr = np.dot(r, z), rr_new
    return x, it, hist


def _edited(module, name, old, new):
    """The function `name` of `module` with one source line replaced (a planted mistake)."""
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(getattr(module, name)))
    assert old in src
    ns = dict(vars(module))
    exec(compile(src.replace(old, new, 1), f"<mutated {name}>", "exec"), ns)
    return ns[name]


def chebyshev_variant(start_width=False, rho_sign=1.0, keep_rho=True):
    def apply(G, minv, r, degree, lmax, ratio):
        a, b = lmax / ratio, lmax
        theta, delta = 0.5 * (b + a), 0.5 * (b - a)
        sigma = theta / delta
        rho = 1.0 / sigma
        d = minv * r / (delta if start_width else theta)
        z = np.zeros_like(r)
        for j in range(degree):
            z = z + d
            if j == degree - 1:
                break
            res = r - G @ z
            rho_next = 1.0 / (2.0 * sigma - rho_sign * rho)
            d = rho_next * (rho if keep_rho else 1.0) * d + (2.0 * rho_next / delta) * (minv * res)
            rho = rho_next
        return z
    return apply


CASES = [
    ("local_D", elements, wrong_D, lambda: th.test_constant_source_gives_zero_velocity_and_exact_pressure(2, 100.0)),
    ("local_S", elements, wrong_S, lambda: tg.test_S_matches_closed_form_integrals(2)),
    ("local_R", elements, wrong_R, lambda: th.test_constant_source_gives_zero_velocity_and_exact_pressure(2, 100.0)),
    ("owner_signs", topology, wrong_signs, lambda: th.test_hybrid_equals_coupled(2, 4, 1.0, 100.0, "none")),
    ("geometry", elements, wrong_geometry_normal, lambda: tg.test_area_normal_is_barycentric_gradient(2)),
    ("local_R_previous", elements, wrong_previous, lambda: tt.test_previous_level_term_is_the_lumped_mass(2, 6)),
    ("local_R_previous", elements, wrong_previous, lambda: tt.test_steady_solution_is_a_fixed_point_of_the_time_step(2, 7)),
    ("minres", krylov, wrong_minres, lambda: tm.test_iterates_equal_scipy_minres(2, 10, 1000.0)),
    ("hybridise", hybrid,
     _edited(hybrid, "hybridise", "M = Ainv - np.einsum(", "M = Ainv + 0.0 * np.einsum("),   # pressure not eliminated
     lambda: th.test_hybrid_equals_coupled(2, 4, 1.0, 100.0, "none")),
    ("hybridise", hybrid,
     _edited(hybrid, "hybridise", "M[k0] = Ainv[k0]", "pass"),                                # K_0 not special-cased
     lambda: th.test_hybrid_equals_coupled(2, 4, 1.0, 100.0, "none")),
    ("pcg", krylov, wrong_pcg, lambda: tk.test_pcg_iterates_equal_scipy_cg(2, 10, 1000.0)),
    ("deflated_pcg", krylov,
     _edited(krylov, "deflated_pcg", "p = project(z) + (rz_new / rz) * p", "p = z + (rz_new / rz) * p"),   # no projection
     lambda: tdf.test_residuals_stay_orthogonal_to_the_vectors()),
    ("lanczos_ritz", krylov,
     _edited(krylov, "lanczos_ritz", "T[j, j + 1] = T[j + 1, j] = -np.sqrt(betas[j]) / alphas[j]",
             "T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]"),               # off-diagonal sign
     lambda: tdf.test_lanczos_matrix_is_q_transpose_g_q()),
    ("lanczos_ritz", krylov,
     _edited(krylov, "lanczos_ritz", "T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)",
             "T[j, j] = 1.0 / alphas[j]"),                                                  # beta/alpha term dropped
     lambda: tdf.test_full_lanczos_gives_the_exact_smallest_eigenvalues()),
    ("lanczos_ritz", krylov,
     _edited(krylov, "lanczos_ritz", "Q.append(z / np.sqrt(rz))", "Q.append(z)"),       # unnormalised vectors
     lambda: tdf.test_lanczos_matrix_is_q_transpose_g_q()),
    ("gmres", krylov, wrong_gmres, lambda: tk.test_gmres_cycle_is_the_minimal_residual_iterate(6)),
    ("chebyshev_apply", krylov, chebyshev_variant(start_width=True), lambda: tc.test_eigenvectors_get_the_closed_form(3)),
    ("chebyshev_apply", krylov, chebyshev_variant(rho_sign=-1.0), lambda: tc.test_eigenvectors_get_the_closed_form(3)),
    ("chebyshev_apply", krylov, chebyshev_variant(keep_rho=False), lambda: tc.test_eigenvectors_get_the_closed_form(3)),
    ("face_mass", steady,
     _edited(steady, "face_mass", "share = geom[\"vol\"] / (d + 1)", "share = geom[\"vol\"] / d"),   # |K|/d
     lambda: ts.test_preconditioner_is_the_transient_coupled_solve(2, 6, "none")),
    ("TransientPreconditioner", steady,
     _edited(steady, "TransientPreconditioner", "SK = Cv * (np.einsum(\"kab,kb->ka\", M, R_K) + u * (gK * invB)[:, None])",
             "SK = Cv * np.einsum(\"kab,kb->ka\", M, R_K)"),                                   # divergence dropped from S
     lambda: ts.test_preconditioner_is_the_transient_coupled_solve(2, 6, "none")),
    ("fgmres", steady,
     _edited(steady, "fgmres", "x = x + Z[:k].T @ y", "x = x + V[:k].T @ y"),            # update from V, not Z
     lambda: ts.test_fgmres_cycle_is_the_minimal_residual_over_span_Z()),
    ("fgmres", steady,
     _edited(steady, "fgmres", "x = x + Z[:k].T @ y", "x = x + V[:k].T @ y"),
     lambda: ts.test_steady_solution_equals_the_direct_solve(2, 10, 1.0, "none", 30.0)),
]


@pytest.mark.parametrize("name,module,bad,pin", CASES, ids=[f"{c[0]}-{i}" for i, c in enumerate(CASES)])
def test_planted_mistake_is_caught(monkeypatch, name, module, bad, pin):
    topology.__dict__["_orig_owner_signs"] = topology.owner_signs
    topology.__dict__["_orig_geometry"] = elements.geometry
    monkeypatch.setattr(module, name, bad)
    with pytest.raises((AssertionError, np.linalg.LinAlgError)), warnings.catch_warnings():
        warnings.simplefilter("ignore")   # e.g. a singular matrix reported by the pin's direct solve
        pin()
