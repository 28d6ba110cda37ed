"""Discretisation sanity pin: manufactured-solution convergence orders.

The paper observes velocity orders tending to 2 and pressure orders above 1
(Section 4.1, Tables 1-3; stored in tests/golden/paper_rates.json).  The
oracle's coupled solve of a manufactured transient Stokes problem on refined
meshes must show the same orders.  A wrong S_K, D_K or R_K term (a dropped
mass or viscous term, a sign) destroys them.
"""

import json
import os

import numpy as np

import synth
from oracle import coupled, pipeline

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_rates.json")))


def errors(dim, n, mu=100.0, nu=1.0):
    coords, elems = synth.mesh2d_square(n) if dim == 2 else synth.mesh3d_kuhn(n)
    ms = synth.manufactured_stokes(dim, mu, nu, pressure=True)
    fbar = synth.element_means(ms["f"], coords, elems, order=6 if dim == 2 else 4)
    sol = pipeline.direct(coords, elems, nu, mu, fbar)
    topo, geom = sol["topo"], sol["geom"]
    xs = coords[topo["face_vertices"]].mean(axis=1)
    eu = np.sqrt(((sol["U"] - ms["u"](xs)) ** 2).sum() / topo["nf"])
    vol = geom["vol"]
    P = coupled.normalise_pressure(sol["P"], vol)
    pe = ms["p"](geom["xK"])
    pe = pe - np.dot(vol, pe) / vol.sum()
    ep = np.sqrt(np.dot(vol, (P - pe) ** 2))
    return eu, ep


def test_golden_table_ratios_are_consistent():
    """The printed orders are log2 ratios of the printed errors (check the fixture)."""
    for key in ("table1_2d_ns", "table2_3d_stokes", "table3_3d_ns"):
        t = GOLDEN[key]
        for col, rcol in (("errl2U", "ratioU"), ("errl2P", "ratioP")):
            e = np.array(t[col])
            r = np.log2(e[:-1] / e[1:])
            assert np.allclose(r, np.array(t[rcol][1:], dtype=float), atol=0.06)


def test_2d_orders():
    E = [errors(2, n) for n in (8, 16, 32)]
    ru = np.log2(E[-2][0] / E[-1][0])
    rp = np.log2(E[-2][1] / E[-1][1])
    assert abs(ru - GOLDEN["asymptotic"]["velocity_order"]) < 0.15
    assert rp > GOLDEN["asymptotic"]["pressure_order_at_least"]


def test_3d_errors_decrease():
    E = [errors(3, n) for n in (2, 4)]
    assert E[1][0] < 0.6 * E[0][0] and E[1][1] < E[0][1]
