"""bench.py's choice of solvers per workload (host logic, no GPU).

The headline (first) solver is the fastest measured one of each workload:
the Chebyshev-preconditioned FP64 PCG in 2D, float-float Jacobi-PCG on the
3D workload, and the Jacobi-preconditioned solvers of the batch and the
Newton step, which do not take the Chebyshev preconditioner.
"""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def parse(monkeypatch, *argv):
    monkeypatch.setattr(sys, "argv", ["bench.py", *argv])
    return bench.parse()


@pytest.mark.parametrize("workload,head", [("cfg2", "fp64_cheb"), ("cfg1", "fp64_cheb"), ("cfg3", "ff"),
                                           ("cfg4", "ff"), ("cfg5", "ff")])
def test_default_headline_per_workload(monkeypatch, workload, head):
    args = parse(monkeypatch, "--workload", workload)
    precs = args.precs.split(",")
    assert precs[0] == head
    assert all(p in bench.PRECS for p in precs)
    if workload in ("cfg4", "cfg5"):
        assert "fp64_cheb" not in precs


def test_explicit_list_is_kept_except_where_unsupported(monkeypatch):
    assert parse(monkeypatch, "--precs", "fp64,ff").precs == "fp64,ff"
    assert parse(monkeypatch, "--workload", "cfg5", "--precs", "fp64_cheb,fp64").precs == "fp64"
    assert parse(monkeypatch, "--workload", "cfg4", "--precs", "fp64_cheb").precs == "ff"


def test_defaults_meet_the_timing_rules(monkeypatch):
    args = parse(monkeypatch)
    assert args.gpus == 1 and args.warmup >= 3 and args.steps >= 1
    assert args.workload == "cfg2" and args.precs.split(",")[0] == "fp64_cheb"
    o = bench.PRECS["fp64_cheb"][0]
    assert o["precond"] == "chebyshev" and o["prec"] == "fp64" and 2 <= o["poly_degree"] <= 16
    assert set(bench.CHEB_RATIO) == {2, 3} and all(r > 1 for r in bench.CHEB_RATIO.values())
