"""The C ABI: the shared library builds for sm_103a, loads without a GPU,
and exports every function that include/msp.h declares.  No compute calls
are made here (they need a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "msp.h")


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"MSP_API\s+[\w\s\*]+?\b(msp_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2508_08702_gb300 import build
    try:
        path = build.build()
    except (RuntimeError, FileNotFoundError) as e:   # no nvcc on this machine
        pytest.skip(f"cannot build the CUDA library here: {e}")
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("msp_build_lattice", "msp_reduce", "msp_enumerate", "msp_solutions"):
        assert required in names
    assert len(names) >= 15


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points(lib):
    from paper_2508_08702_gb300 import msp
    o = msp.msp_opts()
    lib.msp_default_opts(ctypes.byref(o))
    assert (o.N, o.lanes, o.sym, o.hoelder, o.use_eps) == (1024, 0, 1, 0, 1)
    assert abs(o.delta - 0.99) < 1e-15
    lib.msp_status_string.restype = ctypes.c_char_p
    assert lib.msp_status_string(0) == b"ok"
    assert lib.msp_status_string(5).startswith(b"kept vectors")
    # argument checks happen before any device work
    lib.msp_reduce_lattice_noalloc.restype = ctypes.c_int
    assert lib.msp_reduce_lattice_noalloc(0, 5, None, None, 1024, ctypes.c_double(0.99),
                                          ctypes.c_double(0.51), 10, None, None) == 1
