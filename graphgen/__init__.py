"""Seeded synthetic graph generators (C, OpenMP) with a numpy front end.

The generators build the workloads of the hybrid connected-components path:
planted small components, R-MAT scale-free graphs, a percolated grid unioned
with chains, and batches of independent graphs. They hold none of the
connected-components arithmetic. Outputs are interleaved undirected pairs
``edges[m, 2]`` (int32 or int64), plus whatever ground truth the family
plants (component index per vertex for the planted family).

The shared object is compiled on first use with gcc (``build()``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None

_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_dbl = ctypes.c_double
_int = ctypes.c_int
_ptr = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile graphgen.c into libgraphgen.so (skipped if up to date)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.gg_planted_sizes.restype = _i64
        lib.gg_planted_sizes.argtypes = [_u64, _i64, _i64, _dbl, _dbl, _dbl, _ptr]
        lib.gg_planted_fill.restype = None
        lib.gg_planted_fill.argtypes = [_u64, _i64, _i64, _ptr, _dbl, _int, _ptr, _i64, _ptr]
        lib.gg_rmat_fill.restype = None
        lib.gg_rmat_fill.argtypes = [_u64, _int, _i64, _dbl, _dbl, _dbl, _u64, _int, _ptr, _i64]
        lib.gg_gridchain_count.restype = _i64
        lib.gg_gridchain_count.argtypes = [_u64, _i64, _dbl, _i64, _dbl, _dbl, _ptr, _ptr]
        lib.gg_gridchain_fill.restype = None
        lib.gg_gridchain_fill.argtypes = [_u64, _i64, _dbl, _i64, _dbl, _ptr, _i64, _int, _ptr, _i64]
        lib.gg_batch_sizes.restype = None
        lib.gg_batch_sizes.argtypes = [_u64, _i64, _i64, _i64, _int, _dbl, _dbl, _dbl, _ptr, _ptr]
        lib.gg_batch_fill.restype = None
        lib.gg_batch_fill.argtypes = [_u64, _i64, _ptr, _ptr, _int, _dbl, _dbl, _dbl, _dbl, _dbl, _dbl, _ptr]
        lib.gg_batch_fill_ids.restype = None
        lib.gg_batch_fill_ids.argtypes = [_u64, _i64, _ptr, _ptr, _ptr, _dbl, _dbl, _dbl, _dbl, _dbl, _dbl, _ptr]
        lib.gg_permute.restype = None
        lib.gg_permute.argtypes = [_u64, _u64, _u64, _ptr, _ptr, _i64]
        lib.gg_chung_lu_fill.restype = None
        lib.gg_chung_lu_fill.argtypes = [_u64, _i64, _i64, _dbl, _int, _ptr]
        lib.gg_num_threads.restype = _int
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dtype(id_bytes: int):
    if id_bytes not in (4, 8):
        raise ValueError("id_bytes must be 4 or 8")
    return np.int32 if id_bytes == 4 else np.int64


@dataclass
class Graph:
    """An undirected edge list with its vertex count and planted metadata."""

    edges: np.ndarray  # [m, 2] int32 or int64
    n: int
    name: str
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.edges.shape[0])

    @property
    def id_bytes(self) -> int:
        return self.edges.dtype.itemsize


def permute(n: int, seed: int, stream: int, x: np.ndarray) -> np.ndarray:
    """The Feistel id permutation on [0, n) the generators use (for tests)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.uint64)
    out = np.empty_like(x)
    lib.gg_permute(n, seed, stream, _p(x), _p(out), x.size)
    return out


def planted(seed: int = 1, n: int = 65536, ncomp: int = 512, lo: float = 8.0, hi: float = 1024.0,
            extra_per_vertex: float = 1.5, id_bytes: int = 4) -> Graph:
    """K planted components: spanning tree + uniform extra pairs in each.

    ``meta['comp']`` holds the component index of every vertex and
    ``meta['sizes']`` the component sizes (they sum to exactly n).
    """
    lib = _load()
    if ncomp > n:
        raise ValueError("ncomp must be <= n")
    sizes = np.empty(ncomp, dtype=np.int64)
    m = lib.gg_planted_sizes(seed, n, ncomp, lo, hi, extra_per_vertex, _p(sizes))
    edges = np.empty((m, 2), dtype=_dtype(id_bytes))
    comp = np.empty(n, dtype=np.int32)
    lib.gg_planted_fill(seed, n, ncomp, _p(sizes), extra_per_vertex, id_bytes, _p(edges), m, _p(comp))
    return Graph(edges, n, f"planted(n={n},K={ncomp},seed={seed})", {"comp": comp, "sizes": sizes, "ncomp": ncomp})


def rmat(seed: int = 1, scale: int = 24, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         id_bytes: int = 4, m: int | None = None) -> Graph:
    """R-MAT on 2^scale vertices with edge_factor * 2^scale pairs (ids permuted)."""
    lib = _load()
    n = 1 << scale
    if m is None:
        m = edge_factor * n
    edges = np.empty((m, 2), dtype=_dtype(id_bytes))
    lib.gg_rmat_fill(seed, scale, m, a, b, c, 0, id_bytes, _p(edges), 0)
    return Graph(edges, n, f"rmat(scale={scale},ef={edge_factor},seed={seed})",
                 {"scale": scale, "edge_factor": edge_factor, "abc": (a, b, c)})


def grid_chains(seed: int = 1, W: int = 8192, p: float = 0.55, nchains: int = 10_000_000, mean_len: float = 20.0,
                branch_p: float = 0.02, id_bytes: int = 8) -> Graph:
    """W x W bond-percolated grid unioned with disjoint branched chains.

    ``meta['chain_off']`` gives the chain offsets in pre-permutation order;
    every chain is one planted component.
    """
    lib = _load()
    n = ctypes.c_int64(0)
    off = np.empty(nchains + 1, dtype=np.int64)
    m = lib.gg_gridchain_count(seed, W, p, nchains, mean_len, branch_p, ctypes.byref(n), _p(off))
    n = int(n.value)
    if id_bytes == 4 and n >= 2**31:
        raise ValueError("n too large for int32 ids")
    edges = np.empty((m, 2), dtype=_dtype(id_bytes))
    lib.gg_gridchain_fill(seed, W, p, nchains, branch_p, _p(off), n, id_bytes, _p(edges), m)
    return Graph(edges, n, f"grid_chains(W={W},p={p},chains={nchains},seed={seed})",
                 {"W": W, "p": p, "nchains": nchains, "chain_off": off})


def chung_lu(seed: int = 1, n: int = 1 << 20, avg_degree: float = 16.0, alpha: float = 2.5,
             id_bytes: int = 4) -> Graph:
    """Chung-Lu graph with Zipf expected degrees (power-law tail of exponent alpha)."""
    lib = _load()
    m = int(round(n * avg_degree / 2))
    edges = np.empty((m, 2), dtype=_dtype(id_bytes))
    lib.gg_chung_lu_fill(seed, n, m, alpha, id_bytes, _p(edges))
    return Graph(edges, n, f"chung_lu(n={n},avg={avg_degree},alpha={alpha},seed={seed})", {"alpha": alpha})


@dataclass
class Batch:
    """G independent graphs concatenated: local ids, offsets in pairs and vertices."""

    edges: np.ndarray  # [sum m_g, 2] int32, ids local to each graph
    edge_offsets: np.ndarray  # [G+1] int64, in pairs
    vertex_offsets: np.ndarray  # [G+1] int64
    name: str

    @property
    def G(self) -> int:
        return int(self.edge_offsets.size - 1)

    def graph(self, g: int) -> Graph:
        e = self.edges[self.edge_offsets[g]:self.edge_offsets[g + 1]]
        return Graph(e, int(self.vertex_offsets[g + 1] - self.vertex_offsets[g]), f"{self.name}[{g}]")


def batch_sizes(seed: int = 1, G: int = 4096, nmin: int = 1000, nmax: int = 1_000_000, edge_factor: int = 8,
                p: float = 0.55, mean_len: float = 20.0, branch_p: float = 0.02) -> tuple[np.ndarray, np.ndarray]:
    """Vertex and pair counts of every graph of a batch (no pairs drawn)."""
    lib = _load()
    ng = np.empty(G, dtype=np.int64)
    mg = np.empty(G, dtype=np.int64)
    lib.gg_batch_sizes(seed, G, nmin, nmax, edge_factor, p, mean_len, branch_p, _p(ng), _p(mg))
    return ng, mg


def batch(seed: int = 1, G: int = 4096, nmin: int = 1000, nmax: int = 1_000_000, edge_factor: int = 8,
          a: float = 0.57, b: float = 0.19, c: float = 0.19, p: float = 0.55, mean_len: float = 20.0,
          branch_p: float = 0.02, graphs=None) -> Batch:
    """G graphs with log-uniform vertex counts, cycling R-MAT / grid / chain forest.
    `graphs` (graph numbers in [0, G)) keeps only those graphs, in that order,
    each with exactly the pairs it has in the whole batch."""
    lib = _load()
    ng, mg = batch_sizes(seed, G, nmin, nmax, edge_factor, p, mean_len, branch_p)
    gids = np.arange(G, dtype=np.int64) if graphs is None else np.ascontiguousarray(graphs, dtype=np.int64)
    if gids.size and (gids.min() < 0 or gids.max() >= G):
        raise ValueError("graph number outside [0, G)")
    ng, mg = np.ascontiguousarray(ng[gids]), mg[gids]
    eoff = np.zeros(gids.size + 1, dtype=np.int64)
    np.cumsum(mg, out=eoff[1:])
    voff = np.zeros(gids.size + 1, dtype=np.int64)
    np.cumsum(ng, out=voff[1:])
    edges = np.empty((int(eoff[-1]), 2), dtype=np.int32)
    lib.gg_batch_fill_ids(seed, gids.size, _p(gids), _p(ng), _p(eoff), a, b, c, p, mean_len, branch_p, _p(edges))
    sub = "" if graphs is None else f",{gids.size} of them"
    return Batch(edges, eoff, voff, f"batch(G={G},n=[{nmin},{nmax}],seed={seed}{sub})")


def union(parts: list, seed: int = 1, id_bytes: int = 4) -> Graph:
    """Disjoint union of graphs: graph i's ids are shifted past those of
    graphs 0..i-1, then every id goes through one seeded random permutation
    of [0, n) and the pairs are put in a seeded random order, so that no
    component sits in a contiguous id range or a contiguous run of pairs.
    ``meta['comp_of_part']`` gives, per vertex, the part it came from."""
    rng = np.random.default_rng(seed)
    sizes = [int(g.n) for g in parts]
    base = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(base[-1])
    e = np.concatenate([g.edges.astype(np.int64) + base[i] for i, g in enumerate(parts)]) if parts else \
        np.zeros((0, 2), np.int64)
    perm = rng.permutation(n).astype(np.int64)
    e = perm[e][rng.permutation(e.shape[0])]
    part = np.empty(n, dtype=np.int32)
    part[perm] = np.repeat(np.arange(len(parts), dtype=np.int32), sizes)
    return Graph(np.ascontiguousarray(e.astype(_dtype(id_bytes))), n,
                 f"union({len(parts)} parts,seed={seed})", {"comp_of_part": part})


def num_threads() -> int:
    return int(_load().gg_num_threads())
