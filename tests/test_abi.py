"""C-ABI checks that need no GPU: the library loads, exports every function
declared in include/pk.h, and rejects bad arguments with PK_EINVAL before any
CUDA call."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pk():
    import paper_1712_05834_gb300 as pk
    pk.build()
    pk.load()
    return pk


def header_functions():
    src = open(os.path.join(ROOT, "include", "pk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pk_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_function(pk):
    names = header_functions()
    assert "pk_plan" in names and "pk_compute" in names and len(names) >= 10
    lib = ctypes.CDLL(pk.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) <= set(pk.EXPORTED)


def test_config_default(pk):
    c = pk.pk_config_default()
    assert c.box_size == 1000.0 and c.nmesh == 256 and c.window == pk.PK_CIC
    assert c.compensated == 1 and c.interlaced == 0 and c.los_axis == 2
    assert c.poles_mask == 7 and c.batch == 1 and c.subtract_shot == 1
    assert abs(c.dk - 2 * 2 * 3.141592653589793 / 1000.0) < 1e-15


def test_status_strings(pk):
    for s in range(8):
        assert pk.pk_status_string(s).startswith("PK_")
    assert "unknown" in pk.pk_status_string(99)


@pytest.mark.parametrize("field,value,word", [
    ("nmesh", 63, "nmesh"), ("nmesh", 2, "nmesh"), ("nmesh", 8192, "nmesh"),
    ("box_size", 0.0, "box_size"), ("box_size", -1.0, "box_size"),
    ("window", 5, "window"), ("dk", 0.0, "dk"), ("kmin", -0.1, "kmin"),
    ("nmu", -1, "nmu"), ("los_axis", 0, "los_axis"), ("precision", 3, "precision"),
    ("fixed_scale_log2", 50, "fixed_scale_log2"), ("batch", -2, "batch"),
    ("poles_mask", 8, "poles_mask"), ("paint_variant", 2, "paint_variant"),
    ("capacity", -1, "capacity"), ("capacity", 1 << 33, "capacity"),
])
def test_plan_rejects_bad_config(pk, field, value, word):
    c = pk.make_config(1000.0, 64, "cic", dk=0.01)
    setattr(c, field, value)
    with pytest.raises(pk.PkError) as e:
        pk.pk_plan(c)
    assert e.value.status == pk.PK_EINVAL
    assert word in str(e.value)


def test_plan_rejects_empty_binning(pk):
    c = pk.make_config(1000.0, 64, "cic", dk=10.0)
    with pytest.raises(pk.PkError) as e:
        pk.pk_plan(c)
    assert e.value.status == pk.PK_EINVAL


def test_null_arguments(pk):
    lib = pk.load()
    c = pk.make_config(1000.0, 64, "cic", dk=0.01)
    assert lib.pk_plan(ctypes.byref(c), None, None) == pk.PK_EINVAL
    assert lib.pk_paint(None, None, 0, None, 0, 0) == pk.PK_EINVAL
    assert lib.pk_compute(None) == pk.PK_EINVAL
    assert lib.pk_destroy(None) == pk.PK_OK
    assert lib.pk_last_error(None) == b""


def _c_layout(tmp_path, struct, fields):
    """sizeof and offsetof of a header struct, from a gcc-compiled probe."""
    src = tmp_path / "layout.c"
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "pk.h"', "int main(void) {",
             '  printf("%%zu\\n", sizeof(%s));' % struct]
    lines += ['  printf("%%zu\\n", offsetof(%s, %s));' % (struct, f) for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    return int(out[0]), [int(v) for v in out[1:]]


@pytest.mark.parametrize("name", ["pk_config", "pk_result_view", "pk_lognormal_config", "pk_projected_view",
                                  "pk_survey_config", "pk_survey_catalog", "pk_survey_result_view"])
def test_ctypes_structs_match_the_header(pk, tmp_path, name):
    cls = getattr(pk, name)
    fields = [f for f, _ in cls._fields_]
    size, offs = _c_layout(tmp_path, name, fields)
    assert ctypes.sizeof(cls) == size
    assert [getattr(cls, f).offset for f in fields] == offs


def test_config_default_new_fields(pk):
    c = pk.pk_config_default()
    assert c.paint_variant == pk.PK_PAINT_SORT and c.capacity == 0 and c.tile == 0


@pytest.mark.parametrize("field,value,word", [
    ("box_size", 0.0, "box_size"), ("ngrid", 7, "ngrid"), ("ngrid", 2, "ngrid"), ("ngrid", 4096, "ngrid"),
    ("variance", 0.0, "variance"), ("slope", float("nan"), "slope"), ("f_rsd", float("inf"), "f_rsd"),
])
def test_lognormal_plan_rejects_bad_config(pk, field, value, word):
    c = pk.pk_lognormal_config(1000.0, 32, -1.5, 0.0, 1.0, 0.75)
    setattr(c, field, value)
    h = ctypes.c_void_p()
    assert pk.load().pk_lognormal_plan(ctypes.byref(c), None, ctypes.byref(h)) == pk.PK_EINVAL
    assert not h.value
    assert word in pk.load().pk_plan_error().decode()


def test_lognormal_null_arguments(pk):
    lib = pk.load()
    assert lib.pk_lognormal_plan(None, None, None) == pk.PK_EINVAL
    assert lib.pk_lognormal_draw(None, 1, 10, None) == pk.PK_EINVAL
    assert lib.pk_lognormal_field(None, 1, None) == pk.PK_EINVAL
    assert lib.pk_lognormal_destroy(None) == pk.PK_OK


@pytest.mark.parametrize("field,value,word", [
    ("box_size", -1.0, "box_size"), ("nmesh", 7, "nmesh"), ("window", 5, "window"), ("dk", 0.0, "dk"),
    ("poles_mask", 8, "poles_mask"), ("omega_m", 1.5, "omega_m"), ("zmax", -1.0, "zmax"),
    ("p0_fkp", -3.0, "p0_fkp"), ("max_batch", -1, "max_batch"), ("precision", 7, "precision"),
])
def test_survey_plan_rejects_bad_config(pk, field, value, word):
    c = pk.make_survey_config(1000.0, (0.0, 0.0, 0.0), 32)
    setattr(c, field, value)
    h = ctypes.c_void_p()
    assert pk.load().pk_survey_plan(ctypes.byref(c), None, ctypes.byref(h)) == pk.PK_EINVAL
    assert not h.value
    assert word in pk.load().pk_plan_error().decode()


def test_survey_config_default(pk):
    c = pk.pk_survey_config()
    pk.load().pk_survey_config_default(ctypes.byref(c))
    assert c.box_size == 1000.0 and c.nmesh == 256 and c.poles_mask == 7 and c.omega_m == 0.31
    assert list(c.box_origin) == [0.0, 0.0, 0.0] and c.zmax == 5.0 and c.max_batch == 0


def test_survey_null_arguments(pk):
    lib = pk.load()
    assert lib.pk_survey_plan(None, None, None) == pk.PK_EINVAL
    assert lib.pk_survey_paint(None, None, None) == pk.PK_EINVAL
    assert lib.pk_survey_compute(None) == pk.PK_EINVAL
    assert lib.pk_survey_result(None, None) == pk.PK_EINVAL
    assert lib.pk_survey_destroy(None) == pk.PK_OK
    assert lib.pk_survey_launch_count(None) == 0


def test_plan_rejects_too_fine_binning(pk):
    """The bin kernel's FP32 bin estimate is exact to one bin only while
    kmax / dk < 2^20."""
    c = pk.make_config(1000.0, 64, "cic", kmin=0.19, kmax=0.2, dk=1e-7)
    h = ctypes.c_void_p()
    assert pk.load().pk_plan(ctypes.byref(c), None, ctypes.byref(h)) == pk.PK_EINVAL
    assert "too fine" in pk.load().pk_plan_error().decode()


def test_survey_bounds_argument_errors(pk):
    lib = pk.load()
    lo, hi = (ctypes.c_double * 3)(), (ctypes.c_double * 3)()
    assert lib.pk_survey_bounds(None, 0.31, 5.0, None, lo, hi) == pk.PK_EINVAL
    cat = pk.pk_survey_catalog(None, pk.PK_F32, pk.PK_COORD_SKY, None, None, None, 10)
    assert lib.pk_survey_bounds(ctypes.byref(cat), 0.31, 5.0, None, lo, hi) == pk.PK_EINVAL    # NULL pos
    cat = pk.pk_survey_catalog(None, pk.PK_F32, pk.PK_COORD_SKY, None, None, None, 0)
    assert lib.pk_survey_bounds(ctypes.byref(cat), 0.0, 5.0, None, lo, hi) == pk.PK_EINVAL     # no omega_m
    assert lib.pk_survey_bounds(ctypes.byref(cat), 0.31, 5.0, None, lo, hi) == pk.PK_OK        # empty: no GPU call
    assert list(lo) == [float("inf")] * 3 and list(hi) == [float("-inf")] * 3


def test_survey_box_encloses_the_range(pk):
    size, origin = pk.survey_box([0.0, -10.0, 5.0], [100.0, 30.0, 45.0], pad=0.1)
    assert abs(size - 110.0) < 1e-12
    assert np.allclose(origin, [50.0 - 55.0, 10.0 - 55.0, 25.0 - 55.0])
    with pytest.raises(ValueError):
        pk.survey_box([1.0, 1.0, 1.0], [1.0, 1.0, 1.0])
