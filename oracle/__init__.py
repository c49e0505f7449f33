"""CPU oracle for the hybrid connected-components path.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package; the product
path (the CUDA library and its binding) never does, and shares no code with
it.

``cc_oracle.c`` holds the plain definitions (union-find, BFS labeller,
transitive closure, degree distribution, Hurwitz zeta, power-law fit with
the Kolmogorov-Smirnov statistic); ``mlp.py`` holds the route-predictor
network in fp64 numpy. Each function cites the passage of the paper it
follows. The shared object is compiled with gcc on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double
_ptr = ctypes.c_void_p

# Section 3.2 / Table 2: BFS runs iff the K-S statistic is below 0.05.
KS_TAU = 0.05
# Reading of the candidate-xmin rule (the paper defers the fit to an external
# library): a tail needs at least 50 vertices and 3 distinct degree values.
KS_MIN_TAIL = 50
KS_MIN_DISTINCT = 3
# and its range must span a decade: max degree >= 10 * xmin.
KS_MIN_SPAN = 10.0


def build(force: bool = False) -> str:
    """Compile cc_oracle.c into liboracle.so (single threaded, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        for name in ("oracle_uf_labels", "oracle_bfs_labels", "oracle_closure_labels", "oracle_degrees"):
            f = getattr(lib, name)
            f.restype = _int
            f.argtypes = [_ptr, _int, _i64, _i64, _ptr]
        lib.oracle_check_ids.restype = _int
        lib.oracle_check_ids.argtypes = [_ptr, _int, _i64, _i64]
        lib.oracle_max_degree.restype = _i64
        lib.oracle_max_degree.argtypes = [_ptr, _i64]
        lib.oracle_histogram.restype = None
        lib.oracle_histogram.argtypes = [_ptr, _i64, _ptr, _i64]
        lib.oracle_hurwitz_zeta.restype = _dbl
        lib.oracle_hurwitz_zeta.argtypes = [_dbl, _dbl]
        lib.oracle_ks_fit.restype = None
        lib.oracle_ks_fit.argtypes = [_ptr, _i64, _i64, _i64, _dbl, _ptr]
        lib.oracle_multi_bfs.restype = _int
        lib.oracle_multi_bfs.argtypes = [_ptr, _int, _i64, _i64, _ptr, _i64, _i64, _ptr]
        _lib = lib
    return _lib


def _edges(edges: np.ndarray) -> tuple[np.ndarray, int, int]:
    e = np.ascontiguousarray(edges)
    if e.dtype not in (np.int32, np.int64):
        raise TypeError("edges must be int32 or int64")
    if e.size and (e.ndim != 2 or e.shape[1] != 2):
        raise ValueError("edges must have shape [m, 2]")
    return e, e.dtype.itemsize, int(e.size // 2)


def _call_labels(fname: str, edges: np.ndarray, n: int) -> np.ndarray:
    e, w, m = _edges(edges)
    out = np.empty(max(n, 1), dtype=np.int64)
    rc = getattr(_load(), fname)(e.ctypes.data_as(_ptr), w, n, m, out.ctypes.data_as(_ptr))
    if rc == 1:
        raise ValueError("edge id out of range [0, n)")
    if rc != 0:
        raise RuntimeError(f"{fname} failed with code {rc}")
    return out[:n]


def labels_uf(edges: np.ndarray, n: int) -> np.ndarray:
    """Min-id component labels by union-find (Section 1; Fig. 1 caption)."""
    return _call_labels("oracle_uf_labels", edges, n)


def labels_bfs(edges: np.ndarray, n: int) -> np.ndarray:
    """Min-id component labels by one BFS per component, seeds in id order (Section 1)."""
    return _call_labels("oracle_bfs_labels", edges, n)


def labels_closure(edges: np.ndarray, n: int) -> np.ndarray:
    """Min-id component labels from the transitive closure (n <= 256)."""
    if n > 256:
        raise ValueError("closure oracle is for n <= 256")
    return _call_labels("oracle_closure_labels", edges, n)


def cc_labels(edges: np.ndarray, n: int, cross_check: bool | None = None) -> np.ndarray:
    """The oracle's labels: union-find, cross-checked by the BFS labeller.

    ``cross_check`` defaults to on for graphs with at most 2^22 pairs.
    """
    lab = labels_uf(edges, n)
    if cross_check is None:
        cross_check = edges.shape[0] <= (1 << 22)
    if cross_check:
        lab2 = labels_bfs(edges, n)
        if not np.array_equal(lab, lab2):
            raise AssertionError("union-find and BFS labellers disagree")
    return lab


def multi_bfs_distances(edges: np.ndarray, n: int, starts: np.ndarray, cutoff: int = 0) -> np.ndarray:
    """dist[v] = least number of pairs from any start to v (-1: not
    reached), BFS from all starts at once, stopping after `cutoff` levels
    when cutoff > 0 (Section 3.2, the BFS step)."""
    e, w, m = _edges(edges)
    st = np.ascontiguousarray(starts, dtype=np.int64)
    out = np.empty(max(n, 1), dtype=np.int64)
    rc = _load().oracle_multi_bfs(e.ctypes.data_as(_ptr), w, n, m, st.ctypes.data_as(_ptr), st.size, int(cutoff),
                                  out.ctypes.data_as(_ptr))
    if rc == 1:
        raise ValueError("id out of range [0, n)")
    if rc != 0:
        raise RuntimeError(f"oracle_multi_bfs failed with code {rc}")
    return out[:n]


def degrees(edges: np.ndarray, n: int) -> np.ndarray:
    """deg[v] = number of pair endpoints equal to v (Section 3.2, Algorithm 2)."""
    return _call_labels("oracle_degrees", edges, n)


def histogram(deg: np.ndarray) -> np.ndarray:
    """hist[d] = number of vertices of degree d, d in [0, max degree]."""
    deg = np.ascontiguousarray(deg, dtype=np.int64)
    lib = _load()
    mx = int(lib.oracle_max_degree(deg.ctypes.data_as(_ptr), deg.size)) if deg.size else 0
    hist = np.empty(mx + 1, dtype=np.int64)
    lib.oracle_histogram(deg.ctypes.data_as(_ptr), deg.size, hist.ctypes.data_as(_ptr), hist.size)
    return hist


def hurwitz_zeta(s: float, q: float) -> float:
    """Hurwitz zeta(s, q), s > 1, q >= 1, by Euler-Maclaurin summation."""
    return float(_load().oracle_hurwitz_zeta(float(s), float(q)))


def ks_fit(hist: np.ndarray, min_tail: int = KS_MIN_TAIL, min_distinct: int = KS_MIN_DISTINCT,
           min_span: float = KS_MIN_SPAN) -> dict:
    """Discrete power-law fit and K-S statistic over candidate xmin (Section 3.2, Table 2).

    Returns D (the minimum over xmin), alpha and xmin at the minimum, the tail
    size and the number of candidates.
    """
    h = np.ascontiguousarray(hist, dtype=np.int64)
    out = np.zeros(5, dtype=np.float64)
    _load().oracle_ks_fit(h.ctypes.data_as(_ptr), h.size, min_tail, min_distinct, float(min_span),
                          out.ctypes.data_as(_ptr))
    return {"D": float(out[0]), "alpha": float(out[1]), "xmin": int(out[2]), "ntail": int(out[3]),
            "ncand": int(out[4])}


def route_is_bfs(D: float, tau: float = KS_TAU) -> bool:
    """Algorithm 2: run the BFS step iff the K-S statistic is below tau."""
    return D < tau


def log2_buckets(hist: np.ndarray, nbuckets: int = 64) -> np.ndarray:
    """Counts per log2 degree bucket: bucket 0 = degree 0, bucket b = degrees in [2^(b-1), 2^b)."""
    h = np.asarray(hist, dtype=np.int64)
    out = np.zeros(nbuckets, dtype=np.int64)
    for d in np.nonzero(h)[0]:
        b = 0 if d == 0 else int(d).bit_length()
        out[min(b, nbuckets - 1)] += h[d]
    return out
