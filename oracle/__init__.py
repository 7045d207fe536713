"""CPU oracle for the exact Ising degeneracy table g(E,M) and its thermodynamics.

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference leg of ``bench.py`` may import this package. It shares no code with the CUDA path
(``paper_1110_2561_gb300``) and neither imports the other; the two meet only in the seeded
input generators of ``paper_1110_2561_gb300.workloads``, which hold no method arithmetic.

The arithmetic lives in ``isg_oracle.c`` (plain C, built with gcc); this module compiles it and
wraps it with numpy. See the header of ``isg_oracle.c`` for the conventions, each tied to the
passage of Peretyatko et al. (arXiv:1110.2561) it follows:

* ``g_edges``    -- the definition written out: every configuration, every bond (Eq. 1, Sec. 3a).
* ``g_masks``    -- the same table from XOR / NOT / mask / popcount on the configuration word
                    (Sec. 3a-3c), still one configuration at a time; optional OpenMP threads.
* ``g_frontier`` -- an exact dynamic programme over the site order (no 2^N loop), for pinning
                    large lattices.
* ``g_frontier_cut`` -- the same programme for every configuration of a cut set of spins, the
                    rest carrying the cut's fields; for tori whose frontier is too wide.
* ``thermo``     -- Z, <H>, <M>, C, chi from g by the definition of Eq. (2), fp64/long double.
* ``magnetisation`` -- <|M|>, <M^2>, <M^4> and Binder's cumulant from g by the same weights.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "isg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {1: "invalid graph or range", 2: "too large", 3: "out of memory"}


def build(force: bool = False) -> str:
    """Compile isg_oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(path: str):
    lib = ctypes.CDLL(path)
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    f64p = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    lib.oracle_bins.argtypes = [ctypes.c_int, i64, i32p, i32p, i32p, i64p, i64p, i64p]
    lib.oracle_g_edges.argtypes = [ctypes.c_int, i64, i32p, i32p, i32p,
                                   ctypes.c_uint64, ctypes.c_uint64, i64p]
    lib.oracle_g_masks.argtypes = [ctypes.c_int, i64, i32p, i32p, i32p,
                                   ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, i64p]
    lib.oracle_g_frontier.argtypes = [ctypes.c_int, i64, i32p, i32p, i32p, ctypes.c_int, i64p]
    lib.oracle_g_frontier_cut.argtypes = [ctypes.c_int, i64, i32p, i32p, i32p, ctypes.c_uint64, ctypes.c_int,
                                          ctypes.c_int, i64p]
    lib.oracle_thermo.argtypes = [ctypes.c_int, i64, i64, i64p, ctypes.c_int, f64p,
                                  ctypes.c_int, f64p, f64p, f64p, f64p, f64p, f64p]
    lib.oracle_magnetisation.argtypes = [ctypes.c_int, i64, i64, i64p, ctypes.c_int, f64p,
                                         ctypes.c_int, f64p, f64p, f64p, f64p, f64p]
    for f in (lib.oracle_bins, lib.oracle_g_edges, lib.oracle_g_masks, lib.oracle_g_frontier,
              lib.oracle_g_frontier_cut, lib.oracle_thermo, lib.oracle_magnetisation):
        f.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB_PATH)
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _edges(edges):
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int64).reshape(-1, 3))
    return (np.ascontiguousarray(e[:, 0], dtype=np.int32), np.ascontiguousarray(e[:, 1], dtype=np.int32),
            np.ascontiguousarray(e[:, 2], dtype=np.int32))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what}: {ERRORS.get(rc, rc)}")


def bins(n: int, edges, lib=None):
    """(e_min, n_e, n_m) of the table for this graph."""
    lib = lib or _load()
    i, j, J = _edges(edges)
    out = [ctypes.c_int64() for _ in range(3)]
    _check(lib.oracle_bins(n, len(i), _ptr(i, ctypes.c_int32), _ptr(j, ctypes.c_int32),
                           _ptr(J, ctypes.c_int32), *[ctypes.byref(o) for o in out]), "bins")
    return tuple(int(o.value) for o in out)


def _table(n, edges, lib=None):
    e_min, n_e, n_m = bins(n, edges, lib)
    return np.zeros((n_e, n_m), dtype=np.int64)


def g_edges(n: int, edges, s_lo: int = 0, s_hi: int | None = None, lib=None) -> np.ndarray:
    """O0: g over configurations [s_lo, s_hi) by the literal bond loop. Shape (n_e, n+1)."""
    lib = lib or _load()
    i, j, J = _edges(edges)
    g = _table(n, edges, lib)
    s_hi = (1 << n) if s_hi is None else s_hi
    _check(lib.oracle_g_edges(n, len(i), _ptr(i, ctypes.c_int32), _ptr(j, ctypes.c_int32),
                              _ptr(J, ctypes.c_int32), s_lo, s_hi, _ptr(g, ctypes.c_int64)), "g_edges")
    return g


def g_masks(n: int, edges, s_lo: int = 0, s_hi: int | None = None, threads: int = 1, lib=None) -> np.ndarray:
    """O1: g over configurations [s_lo, s_hi) from XOR/NOT/mask/popcount per configuration."""
    lib = lib or _load()
    i, j, J = _edges(edges)
    g = _table(n, edges, lib)
    s_hi = (1 << n) if s_hi is None else s_hi
    _check(lib.oracle_g_masks(n, len(i), _ptr(i, ctypes.c_int32), _ptr(j, ctypes.c_int32),
                              _ptr(J, ctypes.c_int32), s_lo, s_hi, threads, _ptr(g, ctypes.c_int64)),
           "g_masks")
    return g


def g_frontier(n: int, edges, max_active: int = 20, lib=None) -> np.ndarray:
    """Exact g by the frontier dynamic programme (no 2^N loop); raises if the frontier is too wide."""
    lib = lib or _load()
    i, j, J = _edges(edges)
    g = _table(n, edges, lib)
    _check(lib.oracle_g_frontier(n, len(i), _ptr(i, ctypes.c_int32), _ptr(j, ctypes.c_int32),
                                 _ptr(J, ctypes.c_int32), max_active, _ptr(g, ctypes.c_int64)),
           "g_frontier")
    return g


def g_frontier_cut(n: int, edges, cut_mask: int, max_active: int = 20, threads: int = 1, lib=None) -> np.ndarray:
    """Exact g by the frontier programme conditioned on the spins of cut_mask (every cut
    configuration, the rest by a frontier with the cut's fields); for lattices whose own frontier
    is too wide. Raises if the rest's frontier exceeds max_active sites."""
    lib = lib or _load()
    i, j, J = _edges(edges)
    g = _table(n, edges, lib)
    _check(lib.oracle_g_frontier_cut(n, len(i), _ptr(i, ctypes.c_int32), _ptr(j, ctypes.c_int32),
                                     _ptr(J, ctypes.c_int32), cut_mask, max_active, threads, _ptr(g, ctypes.c_int64)),
           "g_frontier_cut")
    return g


def thermo(n: int, e_min: int, g: np.ndarray, T, h, lib=None):
    """logZ, <H>, <M>, C, chi on the grid T x h (arrays of shape (len(T), len(h)))."""
    lib = lib or _load()
    g = np.ascontiguousarray(g, dtype=np.int64)
    T = np.ascontiguousarray(np.atleast_1d(T), dtype=np.float64)
    h = np.ascontiguousarray(np.atleast_1d(h), dtype=np.float64)
    outs = [np.zeros((len(T), len(h)), dtype=np.float64) for _ in range(5)]
    _check(lib.oracle_thermo(n, e_min, g.shape[0], _ptr(g, ctypes.c_int64), len(T), _ptr(T, ctypes.c_double),
                             len(h), _ptr(h, ctypes.c_double), *[_ptr(o, ctypes.c_double) for o in outs]),
           "thermo")
    return tuple(outs)


def magnetisation(n: int, e_min: int, g: np.ndarray, T, h, lib=None):
    """<|M|>, <M^2>, <M^4> and Binder's cumulant on the grid T x h (shape (len(T), len(h)))."""
    lib = lib or _load()
    g = np.ascontiguousarray(g, dtype=np.int64)
    T = np.ascontiguousarray(np.atleast_1d(T), dtype=np.float64)
    h = np.ascontiguousarray(np.atleast_1d(h), dtype=np.float64)
    outs = [np.zeros((len(T), len(h)), dtype=np.float64) for _ in range(4)]
    _check(lib.oracle_magnetisation(n, e_min, g.shape[0], _ptr(g, ctypes.c_int64), len(T),
                                    _ptr(T, ctypes.c_double), len(h), _ptr(h, ctypes.c_double),
                                    *[_ptr(o, ctypes.c_double) for o in outs]), "magnetisation")
    return tuple(outs)


def load_variant(source: str, workdir: str):
    """Compile C source text (a modified copy of isg_oracle.c) in workdir and bind it like the
    oracle. Used by the mutation tests, which plant mistakes in a copy of the oracle to show that
    the pins catch them."""
    src = os.path.join(workdir, "variant.c")
    out = os.path.join(workdir, "libvariant.so")
    with open(src, "w") as f:
        f.write(source)
    subprocess.run(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-o", out, src, "-lm"], check=True)
    return _bind(out)


def source() -> str:
    with open(_SRC) as f:
        return f.read()
