"""Python face of the CPU oracle (test infrastructure only).

Thin ctypes wrapper around oracle/msp_oracle.c.  Only the tests, the smoke
check and the benchmark's CPU-baseline leg may import this module; the CUDA
product path never does.  Every function here follows the paper's steps:

* ``build_lattice``  -- generator matrix of Eq. (2), Sec. 2 (binary bounds)
* ``lll``            -- lattice reduction, Alg. 1 step 1
* ``extract``        -- keep vectors with zero top rows, Alg. 1 step 2
* ``gso``            -- Gram-Schmidt of Eq. (4), Alg. 1 step 3
* ``enumerate``      -- Algorithm 1 (with the readings listed in the C file)
* ``solve``          -- the whole pipeline
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import build as _build

HOELDER_CUT, HOELDER_FILTER, HOELDER_OFF = 0, 1, 2
ERRORS = {0: "ok", 1: "overflow", 2: "iteration cap", 3: "out of memory", 4: "invalid argument"}


class OracleError(RuntimeError):
    pass


class _EnumOpts(C.Structure):
    _fields_ = [("hoelder", C.c_int), ("sym", C.c_int), ("lanes", C.c_int),
                ("use_eps", C.c_int), ("first", C.c_int), ("split_level", C.c_int),
                ("sub_level", C.c_int), ("lds", C.c_int), ("lds_rank", C.c_int)]


class _EnumStats(C.Structure):
    _fields_ = [("nodes", C.c_int64), ("passed", C.c_int64), ("leaves", C.c_int64),
                ("nsol", C.c_int64), ("nprefix", C.c_int64), ("lds_cuts", C.c_int64),
                ("stopped", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.oracle_build_lattice.argtypes = [C.c_int, C.c_int, P, P, C.c_int64, P]
        L.oracle_build_lattice_bounds.argtypes = [C.c_int, C.c_int, P, P, P, C.c_int64, P]
        L.oracle_rmax.argtypes = [C.c_int, P]
        L.oracle_rmax.restype = C.c_int64
        L.oracle_enumerate_bounds.argtypes = [C.c_int, C.c_int, P, P, P, P, C.c_int, C.c_int, P, P, P,
                                              C.POINTER(_EnumOpts), P, P, C.c_int64, P, P, C.c_int64,
                                              C.POINTER(_EnumStats)]
        L.oracle_lll.argtypes = [C.c_int, C.c_int, P, C.c_double, C.c_double, C.c_int64, P, P]
        L.oracle_extract.argtypes = [C.c_int, C.c_int, P, P, P]
        L.oracle_gso.argtypes = [C.c_int, C.c_int, P, P, P, P]
        L.oracle_bkz.argtypes = [C.c_int, C.c_int, P, C.c_int, C.c_double, C.c_int, C.c_int64, P, P, P]
        L.oracle_enumerate.argtypes = [C.c_int, C.c_int, P, P, P, P, C.c_int, C.c_int, P, P,
                                       C.POINTER(_EnumOpts), P, P, C.c_int64, P, P, C.c_int64,
                                       C.POINTER(_EnumStats)]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _check(st: int, what: str):
    if st != 0:
        raise OracleError(f"{what}: {ERRORS.get(st, st)}")


def _bounds(r, n):
    if r is None:
        return None
    r = np.ascontiguousarray(r, dtype=np.int32)
    assert r.shape == (n,)
    return r


def rmax(r) -> int:
    """lcm of the upper bounds (Sec. 2); 1 for binary problems."""
    if r is None:
        return 1
    r = np.ascontiguousarray(r, dtype=np.int32)
    return int(lib().oracle_rmax(len(r), _p(r)))


def build_lattice(A: np.ndarray, d: np.ndarray, N: int = 1024, r=None) -> np.ndarray:
    """Basis vectors of Eq. (2) as rows: shape (n+1, m+n+1), int64.  r: upper
    bounds of x (None: binary)."""
    A = np.ascontiguousarray(A, dtype=np.int32)
    d = np.ascontiguousarray(d, dtype=np.int64)
    m, n = A.shape
    rb = _bounds(r, n)
    basis = np.zeros((n + 1, m + n + 1), dtype=np.int64)
    _check(lib().oracle_build_lattice_bounds(m, n, _p(A), _p(d), _p(rb) if rb is not None else None, N,
                                             _p(basis)), "build_lattice")
    return basis


@dataclass
class LLLResult:
    basis: np.ndarray
    iterations: int
    swaps: int


def lll(basis: np.ndarray, delta: float = 0.99, eta: float = 0.51,
        max_iter: int = 50_000_000) -> LLLResult:
    b = np.ascontiguousarray(basis, dtype=np.int64).copy()
    K, L = b.shape
    it = np.zeros(1, np.int64)
    sw = np.zeros(1, np.int64)
    _check(lib().oracle_lll(K, L, _p(b), delta, eta, max_iter, _p(it), _p(sw)), "lll")
    return LLLResult(b, int(it[0]), int(sw[0]))


def extract(basis: np.ndarray, m: int) -> np.ndarray:
    """Kernel basis: reduced vectors with zero top m entries, top rows dropped."""
    b = np.ascontiguousarray(basis, dtype=np.int64)
    K, L = b.shape
    n = K - 1
    assert L == m + n + 1
    kern = np.zeros((K, n + 1), dtype=np.int32)
    ovf = np.zeros(1, np.int32)
    kept = lib().oracle_extract(m, n, _p(b), _p(kern), _p(ovf))
    if ovf[0]:
        raise OracleError("extract: kept entry outside int32")
    return kern[:kept].copy()


@dataclass
class GSO:
    mu: np.ndarray    # (dd, dd) float64, mu[i][j] for j < i, 1 on the diagonal
    B: np.ndarray     # (dd,) float64 = ||bhat_i||^2
    bhat: np.ndarray  # (dd, dim) float64


def gso(kern: np.ndarray) -> GSO:
    kb = np.ascontiguousarray(kern, dtype=np.int32)
    dd, dim = kb.shape
    mu = np.zeros((dd, dd), np.float64)
    B = np.zeros(dd, np.float64)
    bhat = np.zeros((dd, dim), np.float64)
    _check(lib().oracle_gso(dd, dim, _p(kb), _p(mu), _p(B), _p(bhat)), "gso")
    return GSO(mu, B, bhat)


@dataclass
class BKZResult:
    kern: np.ndarray      # (dd, dim) int32, BKZ-reduced kernel basis
    tours: int
    inserts: int
    nodes: int            # enumeration nodes of the block searches


def bkz(kern: np.ndarray, beta: int, delta: float = 0.99, max_tours: int = 16,
        lll_max_iter: int = 50_000_000) -> BKZResult:
    """BKZ-beta of the kernel basis (Sec. 2; readings in the C file, R14)."""
    b = np.ascontiguousarray(kern, dtype=np.int64).copy()
    dd, dim = b.shape
    t = np.zeros(1, np.int64)
    ins = np.zeros(1, np.int64)
    nd = np.zeros(1, np.int64)
    _check(lib().oracle_bkz(dd, dim, _p(b), beta, delta, max_tours, lll_max_iter, _p(t), _p(ins), _p(nd)), "bkz")
    if np.abs(b).max(initial=0) >= 2 ** 31:
        raise OracleError("bkz: entry outside int32")
    return BKZResult(b.astype(np.int32), int(t[0]), int(ins[0]), int(nd[0]))


@dataclass
class EnumResult:
    nodes: int
    passed: int
    leaves: int
    solutions: np.ndarray        # (count, n) uint8, lexicographically sorted
    nsol: int
    prefixes: Optional[np.ndarray] = None   # (count, dd) int32 (split runs)
    prefix_rho: Optional[np.ndarray] = None
    nprefix: int = 0
    stopped: bool = False
    lds_cuts: int = 0


def sort_solutions(x: np.ndarray) -> np.ndarray:
    if len(x) == 0:
        return x.reshape(0, x.shape[1] if x.ndim == 2 else 0)
    keys = [x[:, c] for c in range(x.shape[1] - 1, -1, -1)]
    return x[np.lexsort(keys)]


def enumerate(kern: np.ndarray, g: GSO, A: np.ndarray, d: np.ndarray, *,
              hoelder: int = HOELDER_CUT, sym: bool = True, lanes: int = 32,
              use_eps: bool = True, first: bool = False,
              split_level: int = -1, sub_level: int = -1,
              prefix: Optional[np.ndarray] = None, lds: int = -1, lds_rank: bool = True, r=None,
              sol_cap: int = 1 << 16, prefix_cap: int = 1 << 20) -> EnumResult:
    """Algorithm 1 over the whole tree, the top part down to ``split_level``
    (recording prefixes), or the subtree below ``prefix`` at ``sub_level``.
    ``lds`` >= 0 runs one limited-discrepancy iteration with that budget;
    ``lds_rank`` picks the discrepancy cost of a value (its position in the
    level's walk, else one for every value after the first; R12)."""
    kb = np.ascontiguousarray(kern, dtype=np.int32)
    A = np.ascontiguousarray(A, dtype=np.int32)
    d = np.ascontiguousarray(d, dtype=np.int64)
    dd, dim = kb.shape
    m, n = A.shape
    o = _EnumOpts(hoelder, int(sym), lanes, int(use_eps), int(first), split_level, sub_level, lds, int(lds_rank))
    pu = np.ascontiguousarray(prefix if prefix is not None else np.zeros(dd), dtype=np.int32)
    sol = np.zeros((sol_cap, max(n, 1)), np.uint8)
    pcap = prefix_cap if split_level >= 0 else 0
    pre_u = np.zeros((max(pcap, 1), dd), np.int32)
    pre_rho = np.zeros(max(pcap, 1), np.float64)
    st = _EnumStats()
    rb = _bounds(r, n)
    _check(lib().oracle_enumerate_bounds(dd, dim, _p(np.ascontiguousarray(g.mu)), _p(np.ascontiguousarray(g.B)),
                                         _p(np.ascontiguousarray(g.bhat)), _p(kb), m, n, _p(A), _p(d),
                                         _p(rb) if rb is not None else None,
                                         C.byref(o), _p(pu), _p(sol), sol_cap, _p(pre_u), _p(pre_rho), pcap,
                                         C.byref(st)), "enumerate")
    if st.nsol > sol_cap:
        raise OracleError(f"enumerate: {st.nsol} solutions exceed sol_cap={sol_cap}")
    if pcap and st.nprefix > pcap:
        raise OracleError(f"enumerate: {st.nprefix} prefixes exceed prefix_cap={pcap}")
    res = EnumResult(nodes=st.nodes, passed=st.passed, leaves=st.leaves,
                     solutions=sort_solutions(sol[:st.nsol].copy()), nsol=int(st.nsol),
                     nprefix=int(st.nprefix), stopped=bool(st.stopped), lds_cuts=int(st.lds_cuts))
    if pcap:
        res.prefixes = pre_u[:st.nprefix].copy()
        res.prefix_rho = pre_rho[:st.nprefix].copy()
    return res


def enumerate_lds(kern: np.ndarray, g: GSO, A: np.ndarray, d: np.ndarray, *, first: bool = False,
                  max_budget: int = 1 << 20, **kw) -> list:
    """Limited discrepancy search: iterations k = 0, 1, 2, ... until one
    reports a solution (first) or no value was held back by the budget (the
    tree is exhausted).  Returns the per-iteration results."""
    out = []
    for k in range(max_budget + 1):
        r = enumerate(kern, g, A, d, first=first, lds=k, **kw)
        out.append(r)
        if (first and r.nsol > 0) or r.lds_cuts == 0:
            break
    return out


@dataclass
class Solved:
    basis: np.ndarray
    kern: np.ndarray
    gso: GSO
    result: EnumResult
    lll_iterations: int


def reduce(A: np.ndarray, d: np.ndarray, N: int = 1024, delta: float = 0.99, r=None):
    """Alg. 1 steps 1-3: lattice of Eq. (2), LLL, extraction, Gram-Schmidt."""
    A = np.ascontiguousarray(A, dtype=np.int32)
    m = A.shape[0]
    red = lll(build_lattice(A, d, N, r=r), delta=delta)
    kern = extract(red.basis, m)
    return red, kern, gso(kern)


def solve(A: np.ndarray, d: np.ndarray, N: int = 1024, delta: float = 0.99, r=None, **kw) -> Solved:
    red, kern, g = reduce(A, d, N, delta, r=r)
    res = enumerate(kern, g, A, d, r=r, **kw)
    return Solved(red.basis, kern, g, res, red.iterations)


def library_path() -> str:
    return os.path.abspath(_build.LIB)
