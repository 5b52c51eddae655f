"""The C ABI: the shared library builds for sm_103a, loads without a GPU,
and exports every function that include/msp.h declares.  The argument
checks that come before any device work are exercised too: bad options,
a NULL context for every entry point that takes one, and context creation
on a machine without a GPU.  No compute calls are made here (they need a
GPU)."""
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


def _bound(lib):
    """The library with the binding's argument and return types."""
    from paper_2508_08702_gb300 import msp
    return msp, msp.load()


def test_option_checks_precede_any_device_call(lib):
    """msp_create validates the options before it touches CUDA, so a bad
    option is MSP_EINVAL (and no context) on any machine."""
    msp, L = _bound(lib)
    out = ctypes.c_void_p(1)
    assert L.msp_create(None, None, None) == msp.MSP_EINVAL
    bad = {"lanes": 3, "warps_per_block": 9, "delta": 1.0, "eta": 0.49, "replicas": 65, "bkz_beta": 1,
           "lds_max": 256, "lds_budget": -2, "hoelder": 3, "N": 0, "max_seconds": 0.0, "lds_rank": 2}
    for k, v in bad.items():
        o = msp.default_opts(**{k: v})
        out = ctypes.c_void_p(1)
        assert L.msp_create(ctypes.byref(out), ctypes.byref(o), None) == msp.MSP_EINVAL, k
        assert out.value is None, k


def test_create_without_a_device_reports_a_cuda_error(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    msp, L = _bound(lib)
    out = ctypes.c_void_p(1)
    assert L.msp_create(ctypes.byref(out), None, None) == msp.MSP_ECUDA
    assert out.value is None


def test_null_context_is_an_error_not_a_crash(lib):
    """Every entry point that takes a context returns MSP_EINVAL for NULL
    (the documented value for the queries) without touching the device."""
    msp, L = _bound(lib)
    n = ctypes.c_size_t(0)
    st = msp.msp_stats()
    E = msp.MSP_EINVAL
    calls = {
        "msp_build_lattice": (None, 1, None, None, None, 0),
        "msp_build_lattice_bounds": (None, 1, None, None, None, None, 0),
        "msp_reduce": (None,),
        "msp_enumerate": (None, 0, 0, 0.0, ctypes.byref(st), None),
        "msp_run_async": (None, 0, 0),
        "msp_wait": (None, None, None),
        "msp_graph_capture": (None, 0, 0),
        "msp_graph_launch": (None,),
        "msp_solutions": (None, 0, None, 0, ctypes.byref(n)),
        "msp_export_gso": (None, 0, None, None, None, None, None),
        "msp_export_reduced": (None, 0, None),
        "msp_export_prefixes": (None, 0, None, None, None, None, 0, ctypes.byref(n), None),
        "msp_phase_ms": (None, None),
        "msp_set_scorer": (None, None),
        "msp_export_features": (None, 0, None, 0, ctypes.byref(n)),
        "msp_mlp_forward": (None, None, None, 0, None),
        "msp_mlp_grad": (None, None, None, None, 1, 1.0, None, None),
        "msp_mlp_train": (None, None, None, None, 1, 1, 1e-3, 1.0, 0, None),
        "msp_fp64_peak": (None, None),
    }
    for name, args in calls.items():
        assert getattr(L, name)(*args) == E, name
    assert L.msp_lanes(None) == 0
    assert L.msp_kernel_launches(None) == 0
    assert L.msp_last_error(None) == b"null context"
    L.msp_destroy(None)
    # every declared function that takes a context is covered above
    ctx_fns = [f for f in declared_functions()
               if re.search(r"\b" + f + r"\s*\(\s*(const\s+)?msp_ctx\s*\*\s*\w+", open(HEADER).read())]
    covered = set(calls) | {"msp_lanes", "msp_kernel_launches", "msp_last_error", "msp_destroy"}
    assert set(ctx_fns) <= covered, sorted(set(ctx_fns) - covered)
