"""CPU checks of the C ABI: libmpm.so builds, loads without a GPU, exports
every entry point include/mpm.h declares, and rejects bad arguments before
touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2602_01723_gb300.build import build
    build()
    from paper_2602_01723_gb300 import _lib
    _lib.lib()
    return _lib


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "mpm.h")).read()
    return sorted(set(re.findall(r"MPM_API\s+[\w\s\*]+?\b(mpm_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("mpm_create", "mpm_load_particles", "mpm_step", "mpm_backward", "mpm_destroy"):
        assert required in names
    assert len(names) >= 16


def test_library_exports_every_declared_symbol(L):
    so = ctypes.CDLL(L.SO)
    for name in declared_symbols():
        assert hasattr(so, name), name
        assert name in L.SIGNATURES, name     # the binding knows its signature


def test_default_options(L):
    o = L.mpm_default_options()
    assert o.n_instances == 1 and o.bound == 3 and o.ckpt_every == 20 and o.scatter == 1
    assert list(o.walls) == [1, 1, 2, 1, 1, 1]


def test_create_rejects_bad_arguments_without_a_device(L):
    lib = L.lib()
    out = ctypes.c_void_p()
    mats = (L.mpm_material * 1)(L.mpm_material(0, 0, 1e4, 0.3, 1.0, 0.0, 30.0))
    g = (ctypes.c_float * 3)(0, -9.8, 0)
    bad_res = [(30, 32, 32), (32, 32, 4), (0, 32, 32)]
    for r in bad_res:
        st = lib.mpm_create((ctypes.c_int32 * 3)(*r), 1 / 32, 1e-4, g, mats, 1, None, ctypes.byref(out))
        assert st == 1 and not out.value          # MPM_ERR_INVALID_ARG, nothing created
    st = lib.mpm_create((ctypes.c_int32 * 3)(32, 32, 32), -1.0, 1e-4, g, mats, 1, None, ctypes.byref(out))
    assert st == 1
    bad = (L.mpm_material * 1)(L.mpm_material(0, 5, 1e4, 0.3, 1.0, 0.0, 30.0))     # unknown plasticity
    st = lib.mpm_create((ctypes.c_int32 * 3)(32, 32, 32), 1 / 32, 1e-4, g, bad, 1, None, ctypes.byref(out))
    assert st == 1
    assert b"material" in lib.mpm_last_error(None)
    assert lib.mpm_destroy(None) == 0            # NULL-safe


def test_entry_points_reject_a_null_context(L):
    lib = L.lib()
    assert lib.mpm_step(None, 1, 0, None) == 1
    assert lib.mpm_sync(None, None) == 1
    assert lib.mpm_backward(None, 0, None, None, None, None, None) == 1
    assert lib.mpm_set_tuning(None, 1, 128, 1) == 1


def test_noalloc_rejects_oversize_grids_before_any_device_work(L):
    lib = L.lib()
    h = np.zeros(64, dtype=np.float32)
    p = ctypes.c_void_p(h.ctypes.data)
    mats = (L.mpm_material * 1)(L.mpm_material(0, 0, 1e4, 0.3, 1.0, 0.0, 30.0))
    st = lib.mpm_substep_noalloc((ctypes.c_int32 * 3)(128, 128, 32), 1 / 128, 1e-4, (ctypes.c_float * 3)(0, -9.8, 0),
                                 mats, 1, None, 1, p, p, p, p, p, p, p, p, p, p, None)
    assert st == 8                                # MPM_ERR_CAPACITY
    st = lib.mpm_substep_noalloc((ctypes.c_int32 * 3)(32, 32, 32), 1 / 32, 1e-4, (ctypes.c_float * 3)(0, -9.8, 0),
                                 mats, 17, None, 1, p, p, p, p, p, p, p, p, p, p, None)
    assert st == 1                                # more than 16 materials


@pytest.mark.parametrize("case", ["nu_half", "nu_minus_one", "negative_bound", "wall_code", "elastic_model",
                                  "plastic_model", "nonfinite_E"])
def test_noalloc_checks_the_table_and_options_like_mpm_create(L, case):
    """The allocation-free entry point rejects, as mpm_create does, a table or
    options that mpm_create rejects, and does so before anything else: on a
    grid too large for its scratch it still answers MPM_ERR_INVALID_ARG, not
    MPM_ERR_CAPACITY."""
    lib = L.lib()
    h = np.zeros(64, dtype=np.float32)
    p = ctypes.c_void_p(h.ctypes.data)
    m = dict(elastic=0, plastic=0, E=1e4, nu=0.3, rho=1.0, ys=0.0, phi=30.0)
    opt = L.mpm_default_options()
    if case == "nu_half":
        m["nu"] = 0.5
    elif case == "nu_minus_one":
        m["nu"] = -1.0
    elif case == "negative_bound":
        opt.bound = -1
    elif case == "wall_code":
        opt.walls[3] = 3
    elif case == "elastic_model":
        m["elastic"] = 2                          # the further models run through mpm_create only
    elif case == "plastic_model":
        m["plastic"] = 3
    elif case == "nonfinite_E":
        m["E"] = float("inf")
    mats = (L.mpm_material * 1)(L.mpm_material(m["elastic"], m["plastic"], m["E"], m["nu"], m["rho"], m["ys"],
                                               m["phi"]))
    big = (ctypes.c_int32 * 3)(128, 128, 32)
    st = lib.mpm_substep_noalloc(big, 1 / 128, 1e-4, (ctypes.c_float * 3)(0, -9.8, 0), mats, 1, ctypes.byref(opt), 1,
                                 p, p, p, p, p, p, p, p, p, p, None)
    assert st == 1, (case, st)                    # MPM_ERR_INVALID_ARG before the capacity check


def test_binding_struct_layouts_match_the_header(L, tmp_path):
    """The ctypes mirrors of mpm_material, mpm_options and mpm_bgdo_options
    have the size and field offsets that a C compiler gives the header's
    declarations (a C program built with gcc prints them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {"mpm_material": L.mpm_material, "mpm_options": L.mpm_options,
               "mpm_bgdo_options": L.mpm_bgdo_options}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mpm.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            a, b, c = line.split()
            got[(a, b)] = int(c)
    for name, cls in structs.items():
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
