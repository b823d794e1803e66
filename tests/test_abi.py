"""The C-ABI library builds, loads and exports every entry point declared in
include/stokes.h (CPU only: no call here touches the GPU)."""

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_stokes_build", os.path.join(ROOT, "paper_2407_01783_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return C.CDLL(b.build())


def declared_functions():
    text = open(os.path.join(ROOT, "include", "stokes.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(stokes_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    from paper_2407_01783_gb300 import _lib as L
    assert sorted(L.EXPORTS) == names


def test_host_only_entry_points(lib):
    from paper_2407_01783_gb300 import _lib as L
    o = L.StokesOptions()
    lib.stokes_default_options(C.byref(o))
    assert o.vcycles == 2 and o.inner_tol == 1e-10 and o.eps_pressure == 1.0
    lib.stokes_status_string.restype = C.c_char_p
    assert lib.stokes_status_string(-8).decode().startswith("incompatible")
    # argument validation happens before any CUDA call
    h = C.c_void_p()
    lib.stokes_setup.argtypes = [C.c_int, C.c_void_p, C.c_double, C.c_double, C.c_double,
                                 C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]
    assert lib.stokes_setup(1, None, 1.0, 1.0, 0.0, None, None, C.byref(h)) == -1
    lib.stokes_destroy.argtypes = [C.c_void_p]
    assert lib.stokes_destroy(None) == 0


def test_options_struct_layout_matches_header():
    """Field order of the ctypes mirror follows the C struct declaration."""
    from paper_2407_01783_gb300 import _lib as L
    text = open(os.path.join(ROOT, "include", "stokes.h")).read()
    body = text[text.index("typedef struct {", text.index("STOKES_PRECISION_MIXED")):]
    body = body[: body.index("} stokes_options;")]
    fields = re.findall(r"\b(?:int|double)\s+([a-z_0-9]+);", body)
    assert fields == [f for f, _ in L.StokesOptions._fields_]


def test_lockstep_and_wait_options_validated_on_host(lib):
    """Defaults of the lockstep-related options, rejection of out-of-range
    values and of bad stokes_solve_multi arguments, all before any CUDA call."""
    import numpy as np
    from paper_2407_01783_gb300 import _lib as L
    o = L.StokesOptions()
    lib.stokes_default_options(C.byref(o))
    assert o.host_wait == 0 and o.vcycle_split == 1
    V = np.zeros((3 ** 3, 3))
    h = C.c_void_p()
    lib.stokes_setup.argtypes = [C.c_int, C.c_void_p, C.c_double, C.c_double, C.c_double,
                                 C.POINTER(L.StokesOptions), C.c_void_p, C.POINTER(C.c_void_p)]
    for field, bad in (("host_wait", 2), ("vcycle_split", 3), ("vcycle_split", -1)):
        ob = L.StokesOptions.from_buffer_copy(o)
        setattr(ob, field, bad)
        assert lib.stokes_setup(2, V.ctypes.data, 1.0, 1.0, 0.0, C.byref(ob), None, C.byref(h)) == -1, field
        assert not h.value
    lib.stokes_solve_multi.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                                       C.c_void_p, C.c_void_p]
    assert lib.stokes_solve_multi(None, 4, None, None, 1e-8, None, None, None) == -1
