"""The C-ABI library: builds, loads without a GPU, exports every entry point
declared in include/tomo.h, and its structs have the layout the binding
assumes.  No compute call is made here."""

import ctypes as C
import os
import re
import subprocess

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "tomo.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tomo_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1103_5904_gb300 import build, tomo
    build.build()
    return tomo.load_library()


def test_every_declared_symbol_is_exported(lib):
    from paper_1103_5904_gb300 import tomo
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(tomo.exported_symbols()) == names


def test_status_strings_and_null_context(lib):
    lib.tomo_status_string.restype = C.c_char_p
    assert lib.tomo_status_string(0) == b"ok"
    assert lib.tomo_status_string(-6) == b"numerical breakdown"
    # NULL context: argument error before any CUDA call
    assert lib.tomo_project(None, None, 1, None, 0, None, None, None, None,
                            None, None) == -1
    assert lib.tomo_backproject(None, None, 1, None, None, None, None, None,
                                None, 0, None) == -1
    assert lib.tomo_solve(None, None, 1, None, None, None, None, None, None,
                          None, C.c_double(0), C.c_double(0), 0, C.c_double(0),
                          0, None, None, None) == -1
    h = C.c_void_p()
    assert lib.tomo_create(C.byref(h), -1) == -1  # invalid device


def test_struct_layout_matches_header(tmp_path):
    from paper_1103_5904_gb300 import tomo
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "tomo.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n",
         sizeof(tomo_cube_geom),
         offsetof(tomo_cube_geom, x0), offsetof(tomo_cube_geom, dz),
         offsetof(tomo_cube_geom, r_obs),
         sizeof(tomo_image_geom), sizeof(tomo_pointing), sizeof(tomo_profile),
         sizeof(tomo_problem), offsetof(tomo_problem, lambda),
         offsetof(tomo_problem, prior_weight_dev), sizeof(tomo_plane_rules),
         sizeof(tomo_tiling), offsetof(tomo_tiling, rules));
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(prog),
                           "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [C.sizeof(tomo.CubeGeom), tomo.CubeGeom.x0.offset,
            tomo.CubeGeom.dz.offset, tomo.CubeGeom.r_obs.offset,
            C.sizeof(tomo.ImageGeom),
            C.sizeof(tomo.Pointing), C.sizeof(tomo.Profile),
            C.sizeof(tomo.Problem), tomo.Problem.lam.offset,
            tomo.Problem.prior_weight_dev.offset, C.sizeof(tomo.PlaneRules),
            C.sizeof(tomo.TilingResult), tomo.TilingResult.rules.offset]
    assert got == want


def test_pointing_columns_match_record_fields():
    """The (n, 12) pointing table of the input generators is read as an array
    of tomo_pointing records: same field order."""
    import synth
    from paper_1103_5904_gb300 import tomo
    assert tuple(n for n, _ in tomo.Pointing._fields_) == synth.POINTING_COLUMNS
