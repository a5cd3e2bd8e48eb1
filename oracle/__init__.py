"""K-truss oracle: test infrastructure only.

Plain, slow, obviously correct CPU implementations of what the K-truss hot path
computes (Blanco, Low, Kim, "Exploration of Fine-Grained Parallelism for Load
Balancing Eager K-truss on GPU and CPU", HPEC 2019).  Only the tests, the
package's smoke check and the benchmark's CPU-baseline leg may import this
package; the product path never does.  It shares no code with the CUDA library.

* ``ktruss``                 Alg. 1 bulk peeling with the eager credit rule of
                             Sec. II-B (plain C, ``oracle.c``).
* ``truss_decomposition``    an independent second algorithm (sequential
                             peeling in support order) giving per-edge
                             trussness (plain C).
* ``edge_support``           support of selected edges inside a kept subgraph,
                             one edge at a time (plain C), for sampled checks of
                             large runs.
* ``triangles``              node-iterator triangle count of a kept subgraph
                             (plain C).
* ``brute.ktruss_dense``     Alg. 1 written literally with dense 0/1 matrices in
                             numpy, for tiny graphs (``oracle/brute.py``).
* ``cpu_f_ktruss``           the paper's fine-grained CPU design (per-edge tasks,
                             atomic supports, zero-terminated rows) with OpenMP
                             (``cpu_f.c``): the multi-core CPU baseline that the
                             benchmark times; checked against ``ktruss``.

Parity pins (what ties the oracle to something other than itself) live in
``tests/test_oracle.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None
_CPUF_SRC = os.path.join(_HERE, "cpu_f.c")
_CPUF_LIB = os.path.join(_HERE, "liboracle_cpuf.so")
_cpuf = None

ERR_INVALID = -1
ERR_NOMEM = -2


def build(force: bool = False) -> str:
    """Compiles oracle.c into liboracle.so with gcc if it is stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def build_cpu_f(force: bool = False) -> str:
    """Compiles cpu_f.c with OpenMP into liboracle_cpuf.so if it is stale."""
    if force or not os.path.exists(_CPUF_LIB) or \
            os.path.getmtime(_CPUF_LIB) < os.path.getmtime(_CPUF_SRC):
        tmp = _CPUF_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _CPUF_SRC])
        os.replace(tmp, _CPUF_LIB)
    return _CPUF_LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        lib.oracle_check_csr.argtypes = [i32, i64, vp, vp]
        lib.oracle_ktruss.argtypes = [i32, i64, vp, vp, i32, vp, vp, vp, vp, i32, vp, vp]
        lib.oracle_truss_decomposition.argtypes = [i32, i64, vp, vp, vp]
        lib.oracle_edge_support.argtypes = [i32, i64, vp, vp, vp, i64, vp, vp]
        lib.oracle_triangles.argtypes = [i32, i64, vp, vp, vp, vp]
        for f in (lib.oracle_check_csr, lib.oracle_ktruss, lib.oracle_truss_decomposition,
                  lib.oracle_edge_support, lib.oracle_triangles):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code}")
        self.code = code


def _csr(row_ptr, col):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    c = np.ascontiguousarray(col, dtype=np.int32)
    return rp, c, rp.shape[0] - 1, c.shape[0]


def _ptr(a):
    return a.ctypes.data if a is not None and a.size else None


@dataclass
class KtrussResult:
    mask: np.ndarray          # uint8[m]
    support: np.ndarray       # int32[m]
    rounds: int
    removed_per_round: list = field(default_factory=list)
    triangles: int = 0
    triangles_per_round: list = field(default_factory=list)


def check_csr(row_ptr, col) -> int:
    rp, c, n, m = _csr(row_ptr, col)
    return int(_load().oracle_check_csr(n, m, _ptr(rp), _ptr(c)))


def ktruss(row_ptr, col, K: int) -> KtrussResult:
    """Alg. 1 with the eager credit rule; see ``oracle_ktruss`` in oracle.c."""
    rp, c, n, m = _csr(row_ptr, col)
    mask = np.zeros(max(m, 1), dtype=np.uint8)
    sup = np.zeros(max(m, 1), dtype=np.int32)
    cap = 4096
    removed = np.zeros(cap, dtype=np.int64)
    tris = np.zeros(cap, dtype=np.int64)
    rounds = ctypes.c_int32(0)
    tri = ctypes.c_int64(0)
    rc = _load().oracle_ktruss(n, m, rp.ctypes.data, _ptr(c), K, mask.ctypes.data, sup.ctypes.data,
                               ctypes.addressof(rounds), removed.ctypes.data, cap,
                               ctypes.addressof(tri), tris.ctypes.data)
    if rc != 0:
        raise OracleError(rc)
    r = rounds.value
    return KtrussResult(mask[:m], sup[:m], r, [int(x) for x in removed[:min(r, cap)]], tri.value,
                        [int(x) for x in tris[:min(r, cap)]])


def truss_decomposition(row_ptr, col) -> np.ndarray:
    """Per-edge trussness by sequential peeling (second algorithm)."""
    rp, c, n, m = _csr(row_ptr, col)
    out = np.zeros(max(m, 1), dtype=np.int32)
    rc = _load().oracle_truss_decomposition(n, m, rp.ctypes.data, _ptr(c), out.ctypes.data)
    if rc != 0:
        raise OracleError(rc)
    return out[:m]


def edge_support(row_ptr, col, queries, keep=None) -> np.ndarray:
    """Support of each queried edge slot inside the subgraph of kept edges."""
    rp, c, n, m = _csr(row_ptr, col)
    q = np.ascontiguousarray(queries, dtype=np.int64)
    out = np.zeros(max(q.shape[0], 1), dtype=np.int64)
    k = None if keep is None else np.ascontiguousarray(keep, dtype=np.uint8)
    rc = _load().oracle_edge_support(n, m, rp.ctypes.data, _ptr(c), _ptr(k), q.shape[0],
                                     _ptr(q), out.ctypes.data)
    if rc != 0:
        raise OracleError(rc)
    return out[:q.shape[0]]


def triangles(row_ptr, col, keep=None) -> int:
    rp, c, n, m = _csr(row_ptr, col)
    k = None if keep is None else np.ascontiguousarray(keep, dtype=np.uint8)
    t = ctypes.c_int64(0)
    rc = _load().oracle_triangles(n, m, rp.ctypes.data, _ptr(c), _ptr(k), ctypes.addressof(t))
    if rc != 0:
        raise OracleError(rc)
    return t.value


def cpu_f_ktruss(row_ptr, col, K: int, threads: int = 0) -> KtrussResult:
    """The paper's fine-grained CPU K-truss (cpu_f.c) on `threads` OpenMP
    threads (0 = the runtime's default, all cores).  Returns mask, support and
    rounds (per-round lists are not recorded)."""
    global _cpuf
    if _cpuf is None:
        lib = ctypes.CDLL(build_cpu_f())
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        lib.cpuf_ktruss.argtypes = [i32, i64, vp, vp, i32, i32, vp, vp, vp]
        lib.cpuf_ktruss.restype = ctypes.c_int
        _cpuf = lib
    rp, c, n, m = _csr(row_ptr, col)
    mask = np.zeros(max(m, 1), dtype=np.uint8)
    sup = np.zeros(max(m, 1), dtype=np.int32)
    rounds = ctypes.c_int32(0)
    rc = _cpuf.cpuf_ktruss(n, m, rp.ctypes.data, _ptr(c), K, threads, mask.ctypes.data,
                           sup.ctypes.data, ctypes.addressof(rounds))
    if rc != 0:
        raise OracleError(rc)
    return KtrussResult(mask[:m], sup[:m], rounds.value)
