"""Seeded synthetic inputs for K-truss: upper-triangular int32 CSR graphs.

Both the CPU oracle and the CUDA library take their inputs from here; this
module holds graph construction only (no triangle, support or pruning
arithmetic).  The heavy generators (G(n, m), R-MAT with planted cliques,
degree-ascending relabel) are plain C in ``graphgen.c``, compiled on first use
with gcc; the small constructive graphs used by closed-form tests are built in
Python from edge lists.

A graph is returned as ``CSR(n, row_ptr, col)`` with ``row_ptr`` int32[n+1] and
``col`` int32[m]: the strictly upper-triangular adjacency of an undirected simple
graph, columns strictly increasing within a row (the input layout of Eager
K-truss, Sec. II-B and Sec. III-D of the paper).

Workload recipes (the synthetic stand-ins for the paper's SNAP graphs):

* ``er(n, m, seed)``: G(n, m), uniform unordered pairs, duplicates rejected.
* ``rmat(scale, edge_factor, seed)``: R-MAT, (a, b, c, d) = (.57, .19, .19, .05),
  no noise, original vertex ids; ``relabel=True`` renumbers vertices by
  ascending degree (ties by id).
* ``rmat(23, 16, 0, n_cliques=64, clique_lo=20, clique_hi=200)``: the R-MAT
  scale-23 graph with 64 planted cliques of sizes 20..200.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from itertools import combinations

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None


@dataclass
class CSR:
    n: int
    row_ptr: np.ndarray  # int32[n+1]
    col: np.ndarray      # int32[m]

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    def rows(self) -> np.ndarray:
        """Source vertex of every edge slot (int32[m])."""
        return np.repeat(np.arange(self.n, dtype=np.int32), np.diff(self.row_ptr))

    def edges(self) -> np.ndarray:
        """(m, 2) int64 array of (row, col) pairs in slot order."""
        return np.stack([self.rows().astype(np.int64), self.col.astype(np.int64)], axis=1)


class _GGCSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int64),
                ("row_ptr", ctypes.POINTER(ctypes.c_int32)),
                ("col", ctypes.POINTER(ctypes.c_int32))]


def build(force: bool = False) -> str:
    """Compiles graphgen.c into libgraphgen.so (gcc, OpenMP) if it is stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_GGCSR)
        lib.gg_er.argtypes = [P, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int]
        lib.gg_rmat.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, ctypes.c_int]
        lib.gg_from_edges.argtypes = [P, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int]
        lib.gg_free.argtypes = [P]
        lib.gg_rand.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.gg_rand.restype = ctypes.c_uint64
        lib.gg_key.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.gg_key.restype = ctypes.c_uint64
        for f in (lib.gg_er, lib.gg_rmat, lib.gg_from_edges):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _take(g: _GGCSR, rc: int) -> CSR:
    lib = _load()
    try:
        if rc != 0:
            raise ValueError(f"graph generator failed with code {rc}")
        n, m = int(g.n), int(g.m)
        rp = np.ctypeslib.as_array(g.row_ptr, shape=(n + 1,)).copy()
        col = (np.ctypeslib.as_array(g.col, shape=(m,)).copy() if m > 0
               else np.zeros(0, dtype=np.int32))
        return CSR(n, rp.astype(np.int32, copy=False), col.astype(np.int32, copy=False))
    finally:
        lib.gg_free(ctypes.byref(g))


def er(n: int, m: int, seed: int, relabel: bool = False) -> CSR:
    """G(n, m) with exactly m distinct undirected edges."""
    g = _GGCSR()
    return _take(g, _load().gg_er(ctypes.byref(g), n, m, seed, int(relabel)))


def _fixed(p: float) -> int:
    return min(int(p * 2.0 ** 64), 2 ** 64 - 1)


def rmat(scale: int, edge_factor: int, seed: int, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, n_cliques: int = 0, clique_lo: int = 20, clique_hi: int = 200,
         relabel: bool = False) -> CSR:
    """R-MAT graph with 2^scale vertices and edge_factor * 2^scale samples."""
    g = _GGCSR()
    rc = _load().gg_rmat(ctypes.byref(g), scale, edge_factor, _fixed(a), _fixed(a + b),
                         _fixed(a + b + c), seed, n_cliques, clique_lo, clique_hi, int(relabel))
    return _take(g, rc)


def from_edges(n: int, edges, relabel: bool = False) -> CSR:
    """Upper-triangular CSR of an undirected edge list (self-loops dropped,
    duplicates merged)."""
    e = np.asarray(list(edges) if not isinstance(edges, np.ndarray) else edges,
                   dtype=np.int32).reshape(-1, 2)
    u = np.ascontiguousarray(e[:, 0])
    v = np.ascontiguousarray(e[:, 1])
    g = _GGCSR()
    rc = _load().gg_from_edges(ctypes.byref(g), n, int(e.shape[0]), u.ctypes.data,
                               v.ctypes.data, int(relabel))
    return _take(g, rc)


def rand_u64(key: int, i: int) -> int:
    """Value i of the counter-based stream ``key`` (SplitMix64 output function)."""
    return int(_load().gg_rand(key, i))


def stream_key(tag: int, seed: int, stream: int) -> int:
    return int(_load().gg_key(tag, seed, stream))


# ------------------------------------------------------------ small graphs

def empty(n: int) -> CSR:
    return CSR(n, np.zeros(n + 1, dtype=np.int32), np.zeros(0, dtype=np.int32))


def complete(n: int) -> CSR:
    """K_n."""
    return from_edges(n, list(combinations(range(n), 2)))


def book(t: int) -> CSR:
    """Book graph B_t: edge (0, 1) plus t vertices adjacent to both."""
    edges = [(0, 1)] + [(0, 2 + j) for j in range(t)] + [(1, 2 + j) for j in range(t)]
    return from_edges(t + 2, edges)


def star(leaves: int) -> CSR:
    return from_edges(leaves + 1, [(0, 1 + j) for j in range(leaves)])


def triangle_strip(L: int) -> CSR:
    """Vertices 0..L-1 with edges (i, i+1) and (i, i+2)."""
    edges = [(i, i + 1) for i in range(L - 1)] + [(i, i + 2) for i in range(L - 2)]
    return from_edges(L, edges)


def disjoint_union(*gs: CSR) -> CSR:
    edges, off = [], 0
    for g in gs:
        e = g.edges() + off
        edges.append(e)
        off += g.n
    e = np.concatenate(edges) if edges else np.zeros((0, 2), dtype=np.int64)
    return from_edges(off, e)


def gnp_small(n: int, p: float, seed: int) -> CSR:
    """Small G(n, p) for exhaustive-style checks: pair (u, v), u < v, is present
    iff draw number (u * n + v) of the seed's stream is below p * 2^64."""
    key = stream_key(4, seed, n)
    thr = _fixed(p)
    edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rand_u64(key, u * n + v) < thr]
    return from_edges(n, edges)


def from_bits(n: int, bits: int) -> CSR:
    """Graph on n vertices whose pair number k (in (0,1), (0,2), ... order) is
    present iff bit k of ``bits`` is set: enumerates all graphs on n vertices."""
    pairs = list(combinations(range(n), 2))
    return from_edges(n, [pr for k, pr in enumerate(pairs) if (bits >> k) & 1])


def relabel_map(n: int, row_ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    """new_id[v] of the degree-ascending relabel (ties by old id), matching
    ``relabel=True`` of the generators."""
    deg = np.bincount(col, minlength=n) + np.diff(row_ptr)
    order = np.lexsort((np.arange(n), deg))
    new = np.empty(n, dtype=np.int64)
    new[order] = np.arange(n)
    return new


# ------------------------------------------------------- named workloads

ER_N, ER_AVG_DEG = 2000, 16


def workload(name: str, seed: int = 0) -> CSR:
    """The named synthetic workloads: 'er2000' (G(2000, 16000)),
    'rmat20' / 'rmat20r' (R-MAT scale 20, ef 16, original ids / relabelled),
    'rmat23c' (R-MAT scale 23, ef 16, 64 planted cliques of sizes 20..200)."""
    if name == "er2000":
        return er(ER_N, ER_N * ER_AVG_DEG // 2, seed)
    if name in ("rmat20", "rmat20r"):
        return rmat(20, 16, seed, relabel=name.endswith("r"))
    if name.startswith("rmat") and name[4:].isdigit():
        return rmat(int(name[4:]), 16, seed)
    if name == "rmat23c":
        return rmat(23, 16, seed, n_cliques=64, clique_lo=20, clique_hi=200)
    raise KeyError(name)


def cached_workload(name: str, seed: int = 0, cache_dir: str | None = None) -> CSR:
    """``workload`` with an on-disk .npy cache (the large R-MAT graphs take
    seconds to generate)."""
    cache_dir = cache_dir or os.path.join(_HERE, "_cache")
    os.makedirs(cache_dir, exist_ok=True)
    base = os.path.join(cache_dir, f"{name}_s{seed}")
    try:
        rp = np.load(base + "_rp.npy")
        col = np.load(base + "_col.npy")
        return CSR(rp.shape[0] - 1, rp, col)
    except (OSError, ValueError):
        g = workload(name, seed)
        np.save(base + "_rp.npy", g.row_ptr)
        np.save(base + "_col.npy", g.col)
        return g


# ------------------------------------------------------------- batches

def _unit(key: int, i: int) -> float:
    """Uniform double in [0, 1) from draw i of stream key (top 53 bits)."""
    return (rand_u64(key, i) >> 11) * (1.0 / 9007199254740992.0)


def batch_config(count: int, seed: int = 0, m_lo: float = 1e3, m_hi: float = 2e6,
                 k_lo: int = 3, k_hi: int = 12):
    """The batching workload: `count` graphs with target sizes log-uniform in
    [m_lo, m_hi] edges.  Even-numbered graphs are G(n, m) with an average
    degree d uniform in [8, 64] and n = max(ceil(2m/d), ceil(2 sqrt(m)) + 1)
    (so that the density stays at most 1/2); odd-numbered graphs are R-MAT
    with scale clamp(ceil(log2(m/16)), 10, 17) and edge factor 16 (their size
    is what that scale gives).  Each graph has a K drawn uniformly from
    [k_lo, k_hi].  Returns a list of (CSR, K)."""
    return _generate(batch_specs(count, seed, m_lo, m_hi, k_lo, k_hi))


def batch_specs(count: int, seed: int = 0, m_lo: float = 1e3, m_hi: float = 2e6,
                k_lo: int = 3, k_hi: int = 12):
    """The (spec, K) pairs of batch_config without building the graphs; graph
    g of the batch is from_spec(spec) of pair g."""
    import math
    key = stream_key(5, seed, count)
    specs = []
    for g in range(count):
        u = _unit(key, 4 * g)
        mt = int(round(math.exp(math.log(m_lo) + u * (math.log(m_hi) - math.log(m_lo)))))
        K = k_lo + int(_unit(key, 4 * g + 1) * (k_hi - k_lo + 1))
        sub_seed = rand_u64(key, 4 * g + 2) & 0x7FFFFFFF
        if g % 2 == 0:
            d = 8.0 + _unit(key, 4 * g + 3) * 56.0
            n = max(int(math.ceil(2 * mt / d)), int(math.ceil(2 * math.sqrt(mt))) + 1)
            specs.append((("er", n, mt, sub_seed), K))
        else:
            scale = min(17, max(10, int(math.ceil(math.log2(max(mt, 1) / 16.0)))))
            specs.append((("rmat", scale, 16, sub_seed), K))
    return specs


def from_spec(spec):
    """The graph of one spec of batch_specs: ("er", n, m, seed) or
    ("rmat", scale, edge_factor, seed)."""
    kind, a, b, sd = spec
    return er(a, b, sd) if kind == "er" else rmat(a, b, sd)


def _generate(specs):
    """Builds the graphs of (spec, K) pairs on a thread pool (the C generator
    releases the GIL); each graph depends only on its own spec."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    _load()
    workers = max(1, min(len(specs), os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        graphs = list(ex.map(from_spec, [sp for sp, _ in specs]))
    return [(g, K) for g, (_, K) in zip(graphs, specs)]


def serve_config(count: int, seed: int = 0, m_lo: float = 1e4, m_hi: float = 5e7,
                 k_lo: int = 3, k_hi: int = 16):
    """The serving workload: `count` requests, each an R-MAT or a G(n, m)
    graph with probability 1/2, target size log-uniform in [m_lo, m_hi] edges
    (same recipes as batch_config), K uniform in [k_lo, k_hi].  Returns a list
    of (CSR, K)."""
    return _generate(serve_specs(count, seed, m_lo, m_hi, k_lo, k_hi))


def serve_specs(count: int, seed: int = 0, m_lo: float = 1e4, m_hi: float = 5e7,
                k_lo: int = 3, k_hi: int = 16):
    """The (spec, K) pairs of serve_config without building the graphs;
    request r is from_spec(spec) of pair r."""
    import math
    key = stream_key(6, seed, count)
    specs = []
    for r in range(count):
        u = _unit(key, 5 * r)
        mt = int(round(math.exp(math.log(m_lo) + u * (math.log(m_hi) - math.log(m_lo)))))
        K = k_lo + int(_unit(key, 5 * r + 1) * (k_hi - k_lo + 1))
        sub_seed = rand_u64(key, 5 * r + 2) & 0x7FFFFFFF
        if _unit(key, 5 * r + 3) < 0.5:
            d = 8.0 + _unit(key, 5 * r + 4) * 56.0
            n = max(int(math.ceil(2 * mt / d)), int(math.ceil(2 * math.sqrt(mt))) + 1)
            specs.append((("er", n, mt, sub_seed), K))
        else:
            scale = min(30, max(10, int(math.ceil(math.log2(max(mt, 1) / 16.0)))))
            specs.append((("rmat", scale, 16, sub_seed), K))
    return specs
