"""The C-ABI library loads and exports every entry point that include/wilson_mg.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_0811_4331_gb300", "libwilsonmg.so")


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "wilson_mg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("mg_", "dslash", "coarse", "restrict", "prolong", "mr_",
                                                         "vcycle", "krylov", "eo_", "schur"))))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_0811_4331_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header(lib):
    from paper_0811_4331_gb300 import wilson_mg
    assert sorted(wilson_mg.EXPORTS) == declared_symbols()


def test_host_only_entry_points(lib):
    """Calls that need no device: defaults, footprint, argument errors."""
    from paper_0811_4331_gb300 import wilson_mg as wm
    p = wm.mg_default_params()
    assert p.n_levels == 2 and p.nu_pre == 2 and p.nu_post == 2 and abs(p.omega - 0.8) < 1e-15
    assert p.gcr_restart == 50 and p.nv[0] == 20 and p.coarse_cycles[0] == 4
    assert wm.mg_footprint((8, 8, 8, 16), p, 1) > 0
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(0, 4, 4, 4)
    st = wm.LIB.mg_setup(ctypes.byref(h), ctypes.c_void_p(1), 0, d, 0.1, ctypes.byref(p), None, None)
    assert st == wm.MG_EINVAL and not h.value
    assert "dims" in wm.mg_last_error()
    # parameters validated before any device work
    d = (ctypes.c_int * 4)(4, 3, 4, 4)
    p.fine_smoother = 1
    st = wm.LIB.mg_setup(ctypes.byref(h), ctypes.c_void_p(1), 0, d, 0.1, ctypes.byref(p), None, None)
    assert st == wm.MG_EINVAL and "even" in wm.mg_last_error()
    p.fine_smoother = 2
    st = wm.LIB.mg_setup(ctypes.byref(h), ctypes.c_void_p(1), 0, (ctypes.c_int * 4)(4, 4, 4, 4), 0.1,
                         ctypes.byref(p), None, None)
    assert st == wm.MG_EINVAL and "fine_smoother" in wm.mg_last_error()
    p.fine_smoother = 0
    p.n_levels = 3
    p.coarse_cycles[0] = 9  # the flexible coarse solver keeps 8 directions
    st = wm.LIB.mg_setup(ctypes.byref(h), ctypes.c_void_p(1), 0, (ctypes.c_int * 4)(8, 8, 8, 8), 0.1,
                         ctypes.byref(p), None, None)
    assert st == wm.MG_EINVAL and "coarse_cycles" in wm.mg_last_error()
    assert wm.LIB.mg_release_work(None, None) == 0
    # null handles and empty batches are refused without touching a device
    assert wm.LIB.mg_solve_many(None, 0, None, None, 1, 1, 1e-10, None, None) == wm.MG_EINVAL
    assert wm.LIB.eo_split(None, 0, None, None, None, 1, None) == wm.MG_EINVAL
    assert wm.LIB.schur_apply(None, 0, None, None, 1, None) == wm.MG_EINVAL
    assert wm.LIB.krylov_solve(None, wm.MG_KRYLOV_BICGSTAB_EO, None, None, 1, 1, 1e-10, 100, None, None) \
        == wm.MG_EINVAL
    ms = (ctypes.c_double * 2)(0.1, 0.2)
    assert wm.LIB.mg_solve_masses(None, ms, None, None, 2, 1, 1e-10, None, None) == wm.MG_EINVAL
    two = (ctypes.c_void_p * 2)(None, None)
    assert wm.LIB.mg_solve_many(two, 2, two, two, 1, 1, 1e-10, None, None) == wm.MG_EINVAL
    assert "distinct and non-null" in wm.mg_last_error()


def test_header_is_plain_c_and_cpp():
    """include/wilson_mg.h compiles as C and as C++ (a C ABI: no C++ types in the declarations)."""
    import shutil
    import subprocess
    hdr = os.path.join(ROOT, "include", "wilson_mg.h")
    for cc, lang in (("gcc", "c"), ("g++", "c++")):
        if not shutil.which(cc):
            pytest.skip(cc + " not available")
        r = subprocess.run([cc, "-fsyntax-only", "-Wall", "-Wextra", "-Werror", "-x", lang, hdr],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
