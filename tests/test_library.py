"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
entry point that include/crhyb.h declares, and rejects invalid meshes in its
host-side topology (these paths run before any CUDA call)."""

import os
import re

import numpy as np
import pytest

from paper_2101_03777_gb300 import build, crhyb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return crhyb.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "crhyb.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cr_[A-Za-z_0-9]+)\s*\(", text)))


def test_every_declared_entry_point_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(crhyb.EXPORTED) == names


@pytest.mark.parametrize("case", ["three_simplices_share_a_face", "index_out_of_range", "flat_simplex",
                                  "no_interior_face"])
def test_invalid_meshes_are_rejected(lib, case):
    if case == "three_simplices_share_a_face":
        coords = np.array([[0, 0], [1, 0], [0, 1], [0, -1], [1, 1]], dtype=np.float64)
        elems = np.array([[0, 1, 2], [0, 1, 3], [0, 1, 4]], dtype=np.int32)
    elif case == "index_out_of_range":
        coords = np.array([[0, 0], [1, 0], [0, 1], [1, 1]], dtype=np.float64)
        elems = np.array([[0, 1, 2], [1, 3, 7]], dtype=np.int32)
    elif case == "flat_simplex":
        coords = np.array([[0, 0], [1, 0], [2, 0], [0, 1]], dtype=np.float64)
        elems = np.array([[0, 1, 2], [0, 1, 3]], dtype=np.int32)
    else:   # two triangles that share only a vertex: every face is on the boundary
        coords = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1]], dtype=np.float64)
        elems = np.array([[0, 1, 2], [0, 3, 4]], dtype=np.int32)
    with pytest.raises(crhyb.CrError) as ei:
        crhyb.cr_mesh_load(coords, elems)
    assert ei.value.name == "CR_ERR_MESH"


def test_bad_arguments_are_rejected(lib):
    with pytest.raises(crhyb.CrError) as ei:
        crhyb.cr_mesh_load(np.zeros((4, 2)), np.zeros((2, 3), dtype=np.int32), k0=5)
    assert ei.value.name == "CR_ERR_ARG"
    # empty meshes: no simplex, or a single one (no interior face can exist)
    for ne in (0, 1):
        with pytest.raises(crhyb.CrError) as ei:
            crhyb.cr_mesh_load(np.array([[0, 0], [1, 0], [0, 1]], dtype=np.float64),
                               np.zeros((ne, 3), dtype=np.int32) + np.arange(3, dtype=np.int32))
        assert ei.value.name == "CR_ERR_ARG"
    # NULL handles of the later entry points
    assert lib.cr_solve_preconditioned(None, 0, None, None, None, None) == -1
    assert lib.cr_system_set_previous(None, None) == -1
    assert lib.cr_solve_batched(None, None, None, None) == -1
    rc = lib.cr_solve(None, 0, None, None, None)
    assert rc == -1 and b"NULL" in lib.cr_last_error()


def test_chebyshev_step_form_query(lib):
    """cr_chebyshev_step_form: the defaults (staged for BF16 values; two rows per
    thread for FP32 values in 3D, one in 2D), CR_ERR_ARG for other arguments, and the
    CRHYB_CHEB_KERNEL override (read once per process, so in a child process)."""
    import subprocess
    import sys
    if os.environ.get("CRHYB_CHEB_KERNEL"):
        pytest.skip("the form is overridden in this environment")
    assert [crhyb.cr_chebyshev_step_form(d, pp) for d in (2, 3) for pp in ("fp32", "bf16")] == \
        ["rows1", "staged", "rows2", "staged"]
    for d, pp in ((1, 1), (4, 2), (2, 0), (3, 3)):
        assert crhyb.CR_ERR[lib.cr_chebyshev_step_form(d, pp)] == "CR_ERR_ARG"
    code = ("from paper_2101_03777_gb300 import crhyb; "
            "print(crhyb.cr_chebyshev_step_form(2, 'fp32'), crhyb.cr_chebyshev_step_form(3, 'bf16'))")
    for form in ("rows1", "rows2", "staged"):
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120,
                             env=dict(os.environ, CRHYB_CHEB_KERNEL=form))
        assert out.returncode == 0, out.stderr
        assert out.stdout.split() == [form, form]
