"""Python binding of the C ABI in include/msp.h (libmsp_gb300.so).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch supplies device memory (for inputs already resident
on the GPU) and the CUDA stream.  There is no CPU fallback: loading fails
loudly when the shared library is missing or no GPU is present.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

MSP_OK, MSP_EINVAL, MSP_ENOMEM, MSP_ECUDA, MSP_EOVERFLOW, MSP_ERANK, MSP_ETIMEOUT, MSP_ETRUNC, \
    MSP_ESTATE, MSP_ECAP, MSP_EQUEUE = range(11)
MSP_ALL, MSP_FIRST = 0, 1
MSP_PLAIN, MSP_LEARNED, MSP_LDS, MSP_LDS_LEARNED = 0, 1, 2, 3
MSP_HOST, MSP_DEVICE = 0, 1


class MspError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: status {status}")
        self.status = status


class msp_opts(C.Structure):
    _fields_ = [("N", C.c_int64), ("delta", C.c_double), ("eta", C.c_double),
                ("lll_max_iter", C.c_int64), ("hoelder", C.c_int), ("sym", C.c_int),
                ("use_eps", C.c_int), ("lanes", C.c_int), ("split_depth", C.c_int),
                ("split_target", C.c_int), ("split_capacity", C.c_int),
                ("warps_per_block", C.c_int), ("blocks_per_sm", C.c_int),
                ("sol_capacity", C.c_int64), ("max_seconds", C.c_double),
                ("donation_capacity", C.c_int64), ("log_features", C.c_int),
                ("lds_budget", C.c_int), ("lds_max", C.c_int), ("first_split_target", C.c_int),
                ("bkz_beta", C.c_int), ("bkz_max_tours", C.c_int), ("replicas", C.c_int),
                ("replica_seed", C.c_uint64), ("lds_rank", C.c_int), ("fuse", C.c_int)]


class msp_stats(C.Structure):
    _fields_ = [("nodes", C.c_int64), ("passed", C.c_int64), ("leaves", C.c_int64),
                ("solutions", C.c_int64), ("prefixes", C.c_int64), ("split_level", C.c_int32),
                ("kernel_rank", C.c_int32), ("lll_iterations", C.c_int64),
                ("lll_swaps", C.c_int64), ("split_nodes", C.c_int64), ("split_passed", C.c_int64),
                ("center_fma", C.c_int64), ("fallbacks", C.c_int64), ("donations", C.c_int64),
                ("walker_util", C.c_double), ("first_ms", C.c_double), ("status", C.c_int32),
                ("lds_budget", C.c_int32),
                ("ms", C.c_double), ("bkz_tours", C.c_int64), ("bkz_inserts", C.c_int64),
                ("bkz_nodes", C.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load libmsp_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is missing: run paper_2508_08702_gb300.build.build()")
    L = C.CDLL(path)
    P = C.c_void_p
    ctx_pp = C.POINTER(C.c_void_p)
    L.msp_default_opts.argtypes = [C.POINTER(msp_opts)]
    L.msp_default_opts.restype = None
    L.msp_create.argtypes = [ctx_pp, C.POINTER(msp_opts), P]
    L.msp_destroy.argtypes = [P]
    L.msp_destroy.restype = None
    L.msp_build_lattice.argtypes = [P, C.c_int, P, P, P, C.c_int]
    L.msp_build_lattice_bounds.argtypes = [P, C.c_int, P, P, P, P, C.c_int]
    L.msp_reduce.argtypes = [P]
    L.msp_enumerate.argtypes = [P, C.c_int, C.c_int, C.c_double, C.POINTER(msp_stats), C.POINTER(msp_stats)]
    L.msp_run_async.argtypes = [P, C.c_int, C.c_int]
    L.msp_wait.argtypes = [P, C.POINTER(msp_stats), C.POINTER(msp_stats)]
    L.msp_solutions.argtypes = [P, C.c_int, P, C.c_size_t, C.POINTER(C.c_size_t)]
    L.msp_export_gso.argtypes = [P, C.c_int, P, P, P, P, P]
    L.msp_export_reduced.argtypes = [P, C.c_int, P]
    L.msp_export_prefixes.argtypes = [P, C.c_int, P, P, P, P, C.c_size_t, C.POINTER(C.c_size_t),
                                      C.POINTER(C.c_int32)]
    L.msp_fp64_peak.argtypes = [P, P]
    L.msp_fp64_peak.restype = C.c_int
    L.msp_phase_ms.argtypes = [P, P]
    L.msp_phase_ms.restype = C.c_int
    L.msp_reduce_lattice_noalloc.argtypes = [C.c_int, C.c_int, P, P, C.c_int64, C.c_double, C.c_double,
                                              C.c_int64, P, P]
    L.msp_reduce_lattice_noalloc.restype = C.c_int
    L.msp_graph_capture.argtypes = [P, C.c_int, C.c_int]
    L.msp_graph_capture.restype = C.c_int
    L.msp_lanes.argtypes = [P]
    L.msp_lanes.restype = C.c_int
    L.msp_graph_launch.argtypes = [P]
    L.msp_graph_launch.restype = C.c_int
    L.msp_mlp_param_count.argtypes = []
    L.msp_mlp_param_count.restype = C.c_int
    L.msp_set_scorer.argtypes = [P, P]
    L.msp_export_features.argtypes = [P, C.c_int, P, C.c_size_t, C.POINTER(C.c_size_t)]
    L.msp_mlp_forward.argtypes = [P, P, P, C.c_int64, P]
    L.msp_mlp_grad.argtypes = [P, P, P, P, C.c_int64, C.c_float, P, P]
    L.msp_mlp_train.argtypes = [P, P, P, P, C.c_int64, C.c_int, C.c_float, C.c_float, C.c_uint64, P]
    for name in ("msp_set_scorer", "msp_export_features", "msp_mlp_forward", "msp_mlp_grad", "msp_mlp_train"):
        getattr(L, name).restype = C.c_int
    L.msp_status_string.argtypes = [C.c_int]
    L.msp_status_string.restype = C.c_char_p
    L.msp_last_error.argtypes = [P]
    L.msp_last_error.restype = C.c_char_p
    L.msp_kernel_launches.argtypes = [P]
    L.msp_kernel_launches.restype = C.c_int64
    for name in ("msp_create", "msp_build_lattice", "msp_reduce", "msp_enumerate", "msp_run_async",
                 "msp_wait", "msp_solutions", "msp_export_gso", "msp_export_reduced",
                 "msp_export_prefixes"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def default_opts(**kw) -> msp_opts:
    o = msp_opts()
    load().msp_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


@dataclass
class Result:
    stats: List[dict]
    total: dict
    status: int


class Context:
    """One msp_ctx: a batch of instances on the current CUDA device."""

    def __init__(self, opts: Optional[msp_opts] = None, stream=None, **kw):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the GB300 library has no CPU path")
        self._L = load()
        self.opts = opts if opts is not None else default_opts(**kw)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        st = self._L.msp_create(C.byref(h), C.byref(self.opts), C.c_void_p(stream.cuda_stream))
        if st != MSP_OK:
            raise MspError(st, "msp_create")
        self._h = h
        self.count = 0
        self.dims = None

    # -- helpers -----------------------------------------------------------
    def _check(self, st: int, what: str, ok=(MSP_OK,)):
        if st not in ok:
            msg = self._L.msp_last_error(self._h).decode()
            raise MspError(st, f"{what} ({self._L.msp_status_string(st).decode()}; {msg})")
        return st

    def close(self):
        if getattr(self, "_h", None):
            self._L.msp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def lanes(self) -> int:
        """Lanes per walker in effect for the current batch (fixes the
        |w|_1 summation order, hence the node counts)."""
        return int(self._L.msp_lanes(self._h))

    @property
    def kernel_launches(self) -> int:
        return int(self._L.msp_kernel_launches(self._h))

    # -- the C ABI -----------------------------------------------------------
    def msp_build_lattice(self, dims: np.ndarray, A, d, r=None):
        """dims (count, 2) int32 on the host; A, d either numpy arrays (host
        memory) or CUDA torch tensors (device memory); r: optional host int32
        upper bounds of x, all instances back to back (None: binary)."""
        dims = np.ascontiguousarray(dims, dtype=np.int32).reshape(-1, 2)
        self.dims = dims
        self.count = len(dims)
        rb = None if r is None else np.ascontiguousarray(r, dtype=np.int32)
        rp = _np_ptr(rb) if rb is not None else None
        self._keep = (A, d, rb)
        if isinstance(A, np.ndarray):
            A = np.ascontiguousarray(A, dtype=np.int32)
            d = np.ascontiguousarray(d, dtype=np.int64)
            self._keep = (A, d, rb)
            st = self._L.msp_build_lattice_bounds(self._h, self.count, _np_ptr(dims), _np_ptr(A), _np_ptr(d), rp,
                                                  MSP_HOST)
        else:
            import torch
            assert A.is_cuda and d.is_cuda and A.dtype == torch.int32 and d.dtype == torch.int64
            assert A.is_contiguous() and d.is_contiguous()
            st = self._L.msp_build_lattice_bounds(self._h, self.count, _np_ptr(dims), C.c_void_p(A.data_ptr()),
                                                  C.c_void_p(d.data_ptr()), rp, MSP_DEVICE)
        self._check(st, "msp_build_lattice")

    def msp_reduce(self):
        self._check(self._L.msp_reduce(self._h), "msp_reduce")

    def _result(self, st, stats, total) -> Result:
        return Result([s.as_dict() for s in stats], total.as_dict(), st)

    def msp_enumerate(self, mode: int = MSP_ALL, order: int = MSP_PLAIN, time_cap_s: float = 0.0,
                      allow=(MSP_OK,)) -> Result:
        stats = (msp_stats * max(self.count, 1))()
        total = msp_stats()
        st = self._L.msp_enumerate(self._h, mode, order, time_cap_s, stats, C.byref(total))
        self._check(st, "msp_enumerate", ok=allow)
        return self._result(st, stats[:self.count], total)

    def msp_run_async(self, mode: int = MSP_ALL, order: int = MSP_PLAIN):
        self._check(self._L.msp_run_async(self._h, mode, order), "msp_run_async")

    def msp_graph_capture(self, mode: int = MSP_ALL, order: int = MSP_PLAIN):
        self._check(self._L.msp_graph_capture(self._h, mode, order), "msp_graph_capture")

    def msp_graph_launch(self):
        self._check(self._L.msp_graph_launch(self._h), "msp_graph_launch")

    def msp_wait(self, allow=(MSP_OK,)) -> Result:
        stats = (msp_stats * max(self.count, 1))()
        total = msp_stats()
        st = self._L.msp_wait(self._h, stats, C.byref(total))
        self._check(st, "msp_wait", ok=allow)
        return self._result(st, stats[:self.count], total)

    # -- subtree scorer ---------------------------------------------------------
    def msp_set_scorer(self, theta):
        """theta: numpy float32 vector of msp_mlp_param_count() entries, or None."""
        if theta is None:
            self._check(self._L.msp_set_scorer(self._h, None), "msp_set_scorer")
            return
        th = np.ascontiguousarray(theta, dtype=np.float32)
        assert th.size == self._L.msp_mlp_param_count()
        self._check(self._L.msp_set_scorer(self._h, _np_ptr(th)), "msp_set_scorer")

    def msp_export_features(self, inst: int) -> np.ndarray:
        cnt = C.c_size_t()
        self._check(self._L.msp_export_features(self._h, inst, None, 0, C.byref(cnt)), "msp_export_features")
        f = np.zeros((max(cnt.value, 1), 32), np.float32)
        self._check(self._L.msp_export_features(self._h, inst, _np_ptr(f), cnt.value, C.byref(cnt)),
                    "msp_export_features")
        return f[:cnt.value]

    def msp_mlp_forward(self, theta, x, y):
        """Device tensors: theta (P,), x (n, 32), y (n, 8) float32."""
        self._check(self._L.msp_mlp_forward(self._h, C.c_void_p(theta.data_ptr()), C.c_void_p(x.data_ptr()),
                                            x.shape[0], C.c_void_p(y.data_ptr())), "msp_mlp_forward")

    def msp_mlp_grad(self, theta, x, target, pos_weight, grad, loss):
        self._check(self._L.msp_mlp_grad(self._h, C.c_void_p(theta.data_ptr()), C.c_void_p(x.data_ptr()),
                                         C.c_void_p(target.data_ptr()), x.shape[0], pos_weight,
                                         C.c_void_p(grad.data_ptr()), C.c_void_p(loss.data_ptr())),
                    "msp_mlp_grad")

    def msp_mlp_train(self, theta, x, target, steps, lr, pos_weight, seed, losses=None):
        self._check(self._L.msp_mlp_train(self._h, C.c_void_p(theta.data_ptr()), C.c_void_p(x.data_ptr()),
                                          C.c_void_p(target.data_ptr()), x.shape[0], steps, lr, pos_weight, seed,
                                          C.c_void_p(losses.data_ptr()) if losses is not None else None),
                    "msp_mlp_train")

    def msp_fp64_peak(self) -> float:
        out = np.zeros(1, np.float64)
        self._check(self._L.msp_fp64_peak(self._h, _np_ptr(out)), "msp_fp64_peak")
        return float(out[0])

    def msp_phase_ms(self) -> dict:
        out = np.zeros(4, np.float64)
        self._check(self._L.msp_phase_ms(self._h, _np_ptr(out)), "msp_phase_ms")
        return dict(reduce=out[0], split=out[1], enumerate=out[2], collect=out[3])

    def msp_solutions(self, inst: int) -> np.ndarray:
        cnt = C.c_size_t()
        self._check(self._L.msp_solutions(self._h, inst, None, 0, C.byref(cnt)), "msp_solutions")
        n = int(self.dims[inst, 1])
        x = np.zeros((max(cnt.value, 1), n), np.uint8)
        st = self._L.msp_solutions(self._h, inst, _np_ptr(x), cnt.value, C.byref(cnt))
        self._check(st, "msp_solutions", ok=(MSP_OK, MSP_ETRUNC))
        return x[:cnt.value]

    def msp_export_gso(self, inst: int):
        dims = np.zeros(2, np.int32)
        self._check(self._L.msp_export_gso(self._h, inst, _np_ptr(dims), None, None, None, None),
                    "msp_export_gso")
        dd, dim = int(dims[0]), int(dims[1])
        kb = np.zeros((dd, dim), np.int32)
        mu = np.zeros((dd, dd), np.float64)
        B = np.zeros(dd, np.float64)
        bhat = np.zeros((dd, dim), np.float64)
        self._check(self._L.msp_export_gso(self._h, inst, _np_ptr(dims), _np_ptr(kb), _np_ptr(mu),
                                           _np_ptr(B), _np_ptr(bhat)), "msp_export_gso")
        return kb, mu, B, bhat

    def msp_export_reduced(self, inst: int) -> np.ndarray:
        m, n = (int(v) for v in self.dims[inst])
        b = np.zeros((n + 1, m + n + 1), np.int64)
        self._check(self._L.msp_export_reduced(self._h, inst, _np_ptr(b)), "msp_export_reduced")
        return b

    def msp_export_prefixes(self, inst: int):
        cnt = C.c_size_t()
        lvl = C.c_int32()
        self._check(self._L.msp_export_prefixes(self._h, inst, None, None, None, None, 0, C.byref(cnt),
                                                C.byref(lvl)), "msp_export_prefixes")
        kb, _, _, _ = self.msp_export_gso(inst)
        dd = kb.shape[0]
        k = max(cnt.value, 1)
        u = np.zeros((k, dd), np.int32)
        rho = np.zeros(k, np.float64)
        nodes = np.zeros(k, np.int64)
        sols = np.zeros(k, np.int32)
        self._check(self._L.msp_export_prefixes(self._h, inst, _np_ptr(u), _np_ptr(rho), _np_ptr(nodes),
                                                _np_ptr(sols), cnt.value, C.byref(cnt), C.byref(lvl)),
                    "msp_export_prefixes")
        c = cnt.value
        return dict(u=u[:c], rho=rho[:c], nodes=nodes[:c], sols=sols[:c], split_level=int(lvl.value))


def msp_reduce_lattice_noalloc(A, d, basis, N: int = 1024, delta: float = 0.99, eta: float = 0.51,
                               max_iter: int = 2_000_000, stream=None) -> int:
    """LLL reduction of one instance into the caller's device buffer `basis`
    ((n+1) x (m+n+1) int64) with no device allocation; A (int32, m x n) and d
    (int64, m) are CUDA tensors.  Returns the msp_status code."""
    import torch
    m, n = A.shape
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(load().msp_reduce_lattice_noalloc(m, n, C.c_void_p(A.data_ptr()), C.c_void_p(d.data_ptr()), N,
                                                 delta, eta, max_iter, C.c_void_p(basis.data_ptr()),
                                                 C.c_void_p(stream.cuda_stream)))


def mlp_param_count() -> int:
    return int(load().msp_mlp_param_count())


def solve(instances: Sequence, mode: int = MSP_ALL, time_cap_s: float = 0.0, allow=(MSP_OK,),
          order: int = MSP_PLAIN, scorer=None, **opts):
    """Build, reduce and enumerate a batch of instances (objects with .A and
    .d); returns (Result, [solutions per instance], Context)."""
    from .instances import pack
    pk = pack(list(instances))
    ctx = Context(**opts)
    if scorer is not None:
        ctx.msp_set_scorer(scorer)
    ctx.msp_build_lattice(pk.dims, pk.A, pk.d, pk.r)
    ctx.msp_reduce()
    res = ctx.msp_enumerate(mode, order, time_cap_s, allow=allow)
    sols = [ctx.msp_solutions(i) for i in range(len(pk.dims))]
    return res, sols, ctx
