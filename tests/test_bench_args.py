"""bench.py's choice of solvers per workload (host logic, no GPU).

The headline (first) solver is the fastest measured one of each workload:
the Chebyshev-preconditioned float-float PCG (its preconditioner steps in FP32
on BF16 values) on the single-system Stokes workloads, and the Jacobi-preconditioned solvers of the batch and the
Newton step, which do not take the Chebyshev preconditioner.  Also the
host-side rules of a bench line: the default workload, the rejection of a step
that missed the tolerance, and the DRAM traffic reported only for the kernel
build it was captured on.
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


@pytest.mark.parametrize("workload,head", [("cfg2", "ff_chebbf"), ("cfg1", "ff_chebbf"), ("cfg3", "ff_chebbf"),
                                           ("cfg4", "ff"), ("cfg5", "ff_chebbf")])
def test_default_headline_per_workload(monkeypatch, workload, head):
    args = parse(monkeypatch, "--workload", workload)
    precs = args.precs.split(",")
    assert precs[0] == head
    assert all(p in bench.PRECS for p in precs)
    if workload == "cfg4":   # the batch runs the Jacobi-preconditioned persistent kernel
        assert not set(precs) & set(bench.CHEB_PRECS)
    if workload == "cfg5":   # Newton steps of several seconds each: two solvers
        assert precs == ["ff_chebbf", "ff"]


def test_explicit_list_is_kept_except_where_unsupported(monkeypatch):
    assert parse(monkeypatch, "--precs", "fp64,ff").precs == "fp64,ff"
    assert parse(monkeypatch, "--workload", "cfg5", "--precs", "fp64_cheb,fp64").precs == "fp64_cheb,fp64"
    assert parse(monkeypatch, "--workload", "cfg4", "--precs", "fp64_cheb").precs == "ff"


def test_defaults_meet_the_timing_rules(monkeypatch):
    """The metric (mixed precision against FP64 at relative residual 1e-10) is quoted on the
    3D 64^3 workload, the largest one-GPU configuration: it is the default, with FP64
    Jacobi-PCG among the timed solvers and the 2D 512^2 workload timed after it."""
    args = parse(monkeypatch)
    assert args.gpus == 1 and args.warmup >= 3 and args.steps >= 1
    assert args.workload == "cfg3" and args.precs.split(",")[0] == "ff_chebbf"
    assert "fp64" in args.precs.split(",") and args.tol == 1e-10
    assert args.also == ["cfg2"] and args.mixed_attempt == 1
    o = bench.PRECS["fp64_cheb"][0]
    assert o["precond"] == "chebyshev" and o["prec"] == "fp64" and 2 <= o["poly_degree"] <= 16
    assert set(bench.CHEB_RATIO) == {2, 3} and all(r > 1 for r in bench.CHEB_RATIO.values())


def test_also_rejects_workloads_it_cannot_time(monkeypatch):
    assert parse(monkeypatch, "--workload", "cfg2").also == []
    assert parse(monkeypatch, "--also", "none").also == []
    with pytest.raises(SystemExit):
        parse(monkeypatch, "--also", "cfg4")


def test_traffic_is_reported_only_for_the_captured_kernel_build(monkeypatch):
    sha = bench.sources_sha("persist")
    assert len(sha) == 64 and sha == bench.sources_sha("persist")
    monkeypatch.setattr(bench, "TRAFFIC", {("cfgX", "ff", None): {"per": "iteration", "bytes": 123.0,
                                                                  "sources": "persist", "sha256": sha}})
    assert bench.measured_traffic("cfgX", "ff") == (123.0, "iteration")
    monkeypatch.setattr(bench, "TRAFFIC", {("cfgX", "ff", None): {"per": "iteration", "bytes": 123.0,
                                                                  "sources": "persist", "sha256": "0" * 64}})
    tb, why = bench.measured_traffic("cfgX", "ff")
    assert tb is None and "changed" in why
    assert bench.measured_traffic("cfgY", "ff")[0] is None


def test_kernel_sections_are_hashed_alone(tmp_path, monkeypatch):
    """A (file, start, end) source hashes the text between its markers: an edit
    outside the section leaves the digest, an edit inside changes it, and a missing
    marker gives None (no capture applies)."""
    csrc = tmp_path / "paper_2101_03777_gb300" / "csrc"
    csrc.mkdir(parents=True)
    f = csrc / "k.cu"
    f.write_text("head\n// <a>\nbody\n// <b>\ntail\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", {"k": [("k.cu", "// <a>", "// <b>")]})
    sha = bench.sources_sha("k")
    f.write_text("HEAD\n// <a>\nbody\n// <b>\nTAIL\n")
    assert bench.sources_sha("k") == sha
    f.write_text("head\n// <a>\nbody2\n// <b>\ntail\n")
    assert bench.sources_sha("k") != sha
    f.write_text("head\nbody\n// <b>\n")
    assert bench.sources_sha("k") is None


def test_every_recorded_kernel_section_exists():
    for key in bench.KERNEL_SOURCES:
        assert bench.sources_sha(key) is not None, key
    for key, t in bench.TRAFFIC.items():
        assert len(key) == 3 and t["sources"] in bench.KERNEL_SOURCES and t["per"] in ("iteration", "launch")


def test_a_step_above_the_tolerance_is_rejected():
    bench.check_step({"status": 0, "relres": 9.9e-11}, 1e-10, "ok")
    with pytest.raises(RuntimeError):
        bench.check_step({"status": 0, "relres": 1.2e-10}, 1e-10, "drifted")
    with pytest.raises(RuntimeError):
        bench.check_step({"status": -4, "relres": 5e-11}, 1e-10, "limit")
