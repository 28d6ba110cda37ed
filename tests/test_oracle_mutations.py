"""Planted mistakes in the oracle must be caught by its pins.

Each case patches one plausible error into the oracle (on the CPU) and runs
the pin that should catch it; the pin has to fail.
"""

import numpy as np
import pytest

from oracle import elements, topology
import test_oracle_geometry as tg
import test_oracle_hybrid as th


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


CASES = [
    ("local_D", elements, wrong_D, lambda: th.test_constant_source_gives_zero_velocity_and_exact_pressure(2, 100.0)),
    ("local_S", elements, wrong_S, lambda: tg.test_S_matches_closed_form_integrals(2)),
    ("local_R", elements, wrong_R, lambda: th.test_constant_source_gives_zero_velocity_and_exact_pressure(2, 100.0)),
    ("owner_signs", topology, wrong_signs, lambda: th.test_hybrid_equals_coupled(2, 4, 1.0, 100.0, "none")),
    ("geometry", elements, wrong_geometry_normal, lambda: tg.test_area_normal_is_barycentric_gradient(2)),
]


@pytest.mark.parametrize("name,module,bad,pin", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_is_caught(monkeypatch, name, module, bad, pin):
    topology.__dict__["_orig_owner_signs"] = topology.owner_signs
    topology.__dict__["_orig_geometry"] = elements.geometry
    monkeypatch.setattr(module, name, bad)
    with pytest.raises((AssertionError, np.linalg.LinAlgError)):
        pin()
