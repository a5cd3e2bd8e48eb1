"""GB300-native fine-grained Eager K-truss.

Python binding of ``libktruss.so`` (C ABI in ``include/ktruss.h``).  This module
only marshals arguments: every step of the K-truss computation runs in the
library's CUDA kernels.  PyTorch provides device memory and the current stream.
There is no CPU fallback: if the library cannot be built or loaded, every call
raises.

    >>> import paper_2009_07929_gb300 as kt
    >>> g = kt.load(row_ptr, col)          # int32 CSR (torch cuda/cpu or numpy)
    >>> mask, support = g.run(3)           # uint8 / int32 cuda tensors
    >>> g.stats()["rounds"]

Method: M. Blanco, T. M. Low, K. Kim, "Exploration of Fine-Grained Parallelism
for Load Balancing Eager K-truss on GPU and CPU", HPEC 2019 (Alg. 1 peeling,
Alg. 3 edge tasks, eager credit rule of Sec. II-B).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBUSY = 0, -1, -2, -3, -4, -5
HOST, DEVICE = 0, 1
KERNEL_BALANCED, KERNEL_EDGE, KERNEL_COARSE, KERNEL_AUTO = 0, 1, 2, 3
UPDATE_NEVER, UPDATE_ALWAYS, UPDATE_AUTO = 0, 1, 2
OPT_SUPPORT_KERNEL, OPT_TIMING, OPT_UPDATE, OPT_LIGHT_MERGE, OPT_SMALL_EDGES = 1, 2, 3, 4, 5
OPT_DEVICE_LOOP, OPT_SUPPORT_SHAPE, OPT_REORDER = 6, 7, 8

_lib = None


class KtrussError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        msg = _lib.ktruss_strerror(code).decode() if _lib is not None else str(code)
        if code == ECUDA and _lib is not None:
            msg += f" (cudaError {_lib.ktruss_last_cuda_error()})"
        super().__init__(f"{what}: {msg} [{code}]" if what else f"{msg} [{code}]")
        self.code = code


class _Stats(ctypes.Structure):
    _fields_ = [
        ("rounds", ctypes.c_int32),
        ("edges_in", ctypes.c_int64),
        ("edges_out", ctypes.c_int64),
        ("triangles_out", ctypes.c_int64),
        ("per_round_len", ctypes.c_int32),
        ("removed_per_round", ctypes.POINTER(ctypes.c_int64)),
        ("live_per_round", ctypes.POINTER(ctypes.c_int64)),
        ("triangles_per_round", ctypes.POINTER(ctypes.c_int64)),
        ("ms_support_per_round", ctypes.POINTER(ctypes.c_float)),
        ("merge_work_per_round", ctypes.POINTER(ctypes.c_int64)),
        ("ms_total", ctypes.c_float),
        ("ms_support", ctypes.c_float),
        ("ms_balance", ctypes.c_float),
        ("ms_prune_compact", ctypes.c_float),
        ("ms_finalize", ctypes.c_float),
        ("support_launches", ctypes.c_int32),
        ("kernel_launches", ctypes.c_int32),
        ("updated_per_round", ctypes.POINTER(ctypes.c_int32)),
        ("ms_update", ctypes.c_float),
        ("ms_device_loop", ctypes.c_float),
        ("device_loop_launches", ctypes.c_int32),
        ("device_loop_rounds", ctypes.c_int32),
    ]


class _Tune(ctypes.Structure):
    _fields_ = [
        ("light_merge", ctypes.c_int32),
        ("small_edges", ctypes.c_int64),
        ("update_mode", ctypes.c_int32),
        ("ms", ctypes.c_float),
        ("trials", ctypes.c_int32),
        ("support_shape", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compiles libktruss.so for sm_103a (in-tree) and returns its path."""
    return _build.build(force=force)


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded libktruss (built first if needed)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.ktruss_load_csr.argtypes = [ctypes.POINTER(vp), i32, i64, vp, vp, ctypes.c_int, vp]
        L.ktruss_run.argtypes = [vp, i32, vp, vp, ctypes.c_int, vp]
        L.ktruss_decompose.argtypes = [vp, vp, vp, ctypes.c_int, vp]
        L.ktruss_load_batch.argtypes = [ctypes.POINTER(vp), i32, vp, i32, i64, vp, vp,
                                        ctypes.c_int, vp]
        L.ktruss_load_batch.restype = ctypes.c_int
        L.ktruss_run_batch.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int, vp]
        L.ktruss_run_batch.restype = ctypes.c_int
        L.ktruss_batch_size.argtypes = [vp, ctypes.POINTER(i32)]
        L.ktruss_batch_size.restype = ctypes.c_int
        L.ktruss_server_create.argtypes = [ctypes.POINTER(vp), i32, i64, i32, i64, vp]
        L.ktruss_server_submit.argtypes = [vp, i32, i64, vp, vp, i32, vp, vp, ctypes.POINTER(i64)]
        L.ktruss_server_step.argtypes = [vp, ctypes.POINTER(i32)]
        L.ktruss_server_take_done.argtypes = [vp, vp, vp, i32, ctypes.POINTER(i32)]
        L.ktruss_server_status.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                           ctypes.POINTER(i64)]
        L.ktruss_server_free.argtypes = [vp]
        L.ktruss_server_set_option.argtypes = [vp, i32, i64]
        L.ktruss_server_free.restype = None
        for f in (L.ktruss_server_create, L.ktruss_server_submit, L.ktruss_server_step,
                  L.ktruss_server_take_done, L.ktruss_server_status, L.ktruss_server_set_option):
            f.restype = ctypes.c_int
        L.ktruss_decompose.restype = ctypes.c_int
        L.ktruss_stats.argtypes = [vp, ctypes.POINTER(_Stats)]
        L.ktruss_set_option.argtypes = [vp, i32, i64]
        L.ktruss_autotune.argtypes = [vp, vp, i32, i32, ctypes.POINTER(_Tune), vp]
        L.ktruss_autotune.restype = ctypes.c_int
        L.ktruss_trim_cache.argtypes = []
        L.ktruss_trim_cache.restype = ctypes.c_int
        L.ktruss_graph_size.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i64)]
        L.ktruss_free.argtypes = [vp]
        L.ktruss_free.restype = None
        L.ktruss_support_noalloc.argtypes = [i32, i64, vp, vp, vp, vp, vp]
        L.ktruss_support_noalloc.restype = ctypes.c_int
        L.ktruss_strerror.argtypes = [ctypes.c_int]
        L.ktruss_strerror.restype = ctypes.c_char_p
        for f in (L.ktruss_load_csr, L.ktruss_run, L.ktruss_stats, L.ktruss_set_option,
                  L.ktruss_graph_size, L.ktruss_last_cuda_error, L.ktruss_version):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != OK:
        raise KtrussError(rc, what)


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _as_i32(a):
    """Returns (pointer, kind, keepalive, length) for an int32 1-D array."""
    if isinstance(a, np.ndarray):
        arr = np.ascontiguousarray(a, dtype=np.int32)
        return arr.ctypes.data if arr.size else None, HOST, arr, arr.shape[0]
    torch = _torch()
    if isinstance(a, torch.Tensor):
        t = a.contiguous()
        if t.dtype != torch.int32:
            t = t.to(torch.int32)
        kind = DEVICE if t.is_cuda else HOST
        return (t.data_ptr() if t.numel() else None), kind, t, t.shape[0]
    arr = np.ascontiguousarray(np.asarray(a), dtype=np.int32)
    return arr.ctypes.data if arr.size else None, HOST, arr, arr.shape[0]


@dataclass
class Stats:
    rounds: int
    edges_in: int
    edges_out: int
    triangles_out: int
    removed_per_round: list
    live_per_round: list
    triangles_per_round: list
    ms_support_per_round: list
    merge_work_per_round: list
    ms_total: float
    ms_support: float
    ms_balance: float
    ms_prune_compact: float
    ms_finalize: float
    support_launches: int
    kernel_launches: int
    updated_per_round: list
    ms_update: float
    ms_device_loop: float
    device_loop_launches: int
    device_loop_rounds: int

    def __getitem__(self, k):
        return getattr(self, k)


class Graph:
    """A CSR graph resident on the current CUDA device (ktruss_load_csr)."""

    def __init__(self, handle: int, n: int, m: int):
        self._h = ctypes.c_void_p(handle)
        self.n, self.m = n, m

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ktruss_free(self._h)
            self._h = ctypes.c_void_p(0)

    def set_option(self, key: int, value: int):
        _check(lib().ktruss_set_option(self._h, key, value), "ktruss_set_option")

    def set_kernel(self, kernel: int):
        self.set_option(OPT_SUPPORT_KERNEL, kernel)

    def autotune(self, K, reps: int = 2, stream=None) -> dict:
        """ktruss_autotune: times whole runs of this graph (K an int) or batch
        (K one value per graph) with candidate support-kernel CTA shapes,
        light-merge thresholds, AUTO kernel thresholds and update modes,
        leaves the fastest set on the handle and returns them."""
        Ks = np.ascontiguousarray(np.atleast_1d(np.asarray(K, dtype=np.int32)))
        t = _Tune()
        _check(lib().ktruss_autotune(self._h, Ks.ctypes.data, Ks.shape[0], reps, ctypes.byref(t),
                                     _stream_ptr(stream)), "ktruss_autotune")
        return {"light_merge": t.light_merge, "small_edges": t.small_edges,
                "update_mode": t.update_mode, "support_shape": t.support_shape, "ms": t.ms,
                "trials": t.trials}

    def set_update(self, mode: int):
        """UPDATE_NEVER (recompute S every round, Alg. 1 as written),
        UPDATE_ALWAYS or UPDATE_AUTO (default): see KTRUSS_OPT_UPDATE."""
        self.set_option(OPT_UPDATE, mode)

    def set_support_shape(self, shape: int):
        """KTRUSS_OPT_SUPPORT_SHAPE: 0 = 1024-thread CTAs with 8192-slot
        stages, 1 (default) = 512-thread CTAs, three per SM, 2048-slot
        stages."""
        self.set_option(OPT_SUPPORT_SHAPE, shape)

    def set_reorder(self, on: bool):
        """KTRUSS_OPT_REORDER: runs start from the vertices renumbered by
        ascending degree at load (True, default for single graphs) or from the
        loaded numbering; outputs are in input edge order either way."""
        self.set_option(OPT_REORDER, 1 if on else 0)

    def set_device_loop(self, on: bool):
        """KTRUSS_OPT_DEVICE_LOOP: rounds whose supports come from the update
        run in the device-driven loop (True, default) or from the host."""
        self.set_option(OPT_DEVICE_LOOP, 1 if on else 0)

    def run(self, K: int, support: bool = True, out=None, stream=None):
        """K-truss on the device (ktruss_run, device outputs on the current
        torch stream).  Returns (mask uint8[m], support int32[m] or None)."""
        torch = _torch()
        dev = torch.device("cuda", torch.cuda.current_device())
        if out is not None:
            mask, sup = out
        else:
            mask = torch.empty(max(self.m, 1), dtype=torch.uint8, device=dev)[: self.m]
            sup = (torch.empty(max(self.m, 1), dtype=torch.int32, device=dev)[: self.m]
                   if support else None)
        rc = lib().ktruss_run(self._h, K, mask.data_ptr() if self.m else None,
                              sup.data_ptr() if (sup is not None and self.m) else None, DEVICE,
                              _stream_ptr(stream))
        _check(rc, "ktruss_run")
        return mask, sup

    def run_host(self, K: int, support: bool = True, mask_out=None, support_out=None,
                 stream=None):
        """K-truss with host output buffers (numpy, pageable or pinned torch)."""
        if mask_out is None:
            mask_out = np.zeros(self.m, dtype=np.uint8)
        if support_out is None and support:
            support_out = np.zeros(self.m, dtype=np.int32)

        def ptr(a):
            if a is None or self.m == 0:
                return None
            return a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr()

        rc = lib().ktruss_run(self._h, K, ptr(mask_out), ptr(support_out), HOST,
                              _stream_ptr(stream))
        _check(rc, "ktruss_run")
        return mask_out, support_out

    def decompose(self, out=None, stream=None):
        """Truss decomposition (ktruss_decompose) on the device: returns
        (trussness int32[m] cuda tensor, K_max)."""
        torch = _torch()
        dev = torch.device("cuda", torch.cuda.current_device())
        tr = out if out is not None else torch.empty(max(self.m, 1), dtype=torch.int32,
                                                     device=dev)[: self.m]
        kmax = ctypes.c_int32(0)
        rc = lib().ktruss_decompose(self._h, tr.data_ptr() if self.m else None,
                                    ctypes.addressof(kmax), DEVICE, _stream_ptr(stream))
        _check(rc, "ktruss_decompose")
        return tr, kmax.value

    def run_batch(self, K, support: bool = True, out=None, stream=None):
        """Batched K-truss (ktruss_run_batch), graph k with K[k]; device
        outputs on the current torch stream.  Returns (mask, support, rounds)
        with rounds a numpy int32[G]."""
        torch = _torch()
        G = ctypes.c_int32(0)
        _check(lib().ktruss_batch_size(self._h, ctypes.byref(G)), "ktruss_batch_size")
        Ks = np.ascontiguousarray(np.broadcast_to(np.asarray(K, dtype=np.int32), (G.value,)))
        dev = torch.device("cuda", torch.cuda.current_device())
        if out is not None:
            mask, sup = out
        else:
            mask = torch.empty(max(self.m, 1), dtype=torch.uint8, device=dev)[: self.m]
            sup = (torch.empty(max(self.m, 1), dtype=torch.int32, device=dev)[: self.m]
                   if support else None)
        rounds = np.zeros(G.value, dtype=np.int32)
        rc = lib().ktruss_run_batch(self._h, Ks.ctypes.data, mask.data_ptr() if self.m else None,
                                    sup.data_ptr() if (sup is not None and self.m) else None,
                                    rounds.ctypes.data, DEVICE, _stream_ptr(stream))
        _check(rc, "ktruss_run_batch")
        return mask, sup, rounds

    def stats(self) -> Stats:
        st = _Stats()
        _check(lib().ktruss_stats(self._h, ctypes.byref(st)), "ktruss_stats")
        r = st.per_round_len

        def arr(p, typ=int):
            return [typ(p[i]) for i in range(r)] if r else []

        return Stats(st.rounds, st.edges_in, st.edges_out, st.triangles_out,
                     arr(st.removed_per_round), arr(st.live_per_round),
                     arr(st.triangles_per_round), arr(st.ms_support_per_round, float),
                     arr(st.merge_work_per_round),
                     st.ms_total, st.ms_support, st.ms_balance, st.ms_prune_compact,
                     st.ms_finalize, st.support_launches, st.kernel_launches,
                     arr(st.updated_per_round), st.ms_update, st.ms_device_loop,
                     st.device_loop_launches, st.device_loop_rounds)


def load(row_ptr, col, stream=None) -> Graph:
    """Copies an upper-triangular int32 CSR (torch cuda/cpu tensors or numpy
    arrays; both of the same kind) into a new graph handle (ktruss_load_csr)."""
    rp_p, rp_kind, rp_keep, rp_len = _as_i32(row_ptr)
    c_p, c_kind, c_keep, m = _as_i32(col)
    if m > 0 and rp_kind != c_kind:
        raise ValueError("row_ptr and col must both be host or both be device arrays")
    n = rp_len - 1
    if n < 0:
        raise KtrussError(EINVAL, "ktruss_load_csr")
    h = ctypes.c_void_p(0)
    rc = lib().ktruss_load_csr(ctypes.byref(h), n, m, rp_p, c_p, rp_kind, _stream_ptr(stream))
    _check(rc, "ktruss_load_csr")
    return Graph(h.value, n, m)


def concat_graphs(graphs):
    """Block-diagonal concatenation of CSR graphs (objects with n, row_ptr,
    col): returns (vertex_offsets int32[G+1], row_ptr int32[n+1], col int32[m],
    edge_offsets int64[G+1]) with global vertex ids."""
    ns = [int(g.n) for g in graphs]
    ms = [int(np.asarray(g.col).shape[0]) for g in graphs]
    vo = np.zeros(len(graphs) + 1, dtype=np.int64)
    vo[1:] = np.cumsum(ns)
    eo = np.zeros(len(graphs) + 1, dtype=np.int64)
    eo[1:] = np.cumsum(ms)
    if vo[-1] >= 2 ** 31 or eo[-1] >= 2 ** 31:
        raise ValueError("batch too large for int32 CSR indices")
    rp = np.zeros(int(vo[-1]) + 1, dtype=np.int32)
    col = np.zeros(int(eo[-1]), dtype=np.int32)
    for k, g in enumerate(graphs):
        r = np.asarray(g.row_ptr, dtype=np.int64)
        rp[vo[k] + 1: vo[k + 1] + 1] = (r[1:] + eo[k]).astype(np.int32)
        col[eo[k]: eo[k + 1]] = (np.asarray(g.col, dtype=np.int64) + vo[k]).astype(np.int32)
    return vo.astype(np.int32), rp, col, eo


def load_batch(graphs=None, vertex_offsets=None, row_ptr=None, col=None, stream=None) -> Graph:
    """ktruss_load_batch: either a list of CSR graphs (concatenated here), or a
    prepared block-diagonal CSR with its vertex offsets (host int32[G+1])."""
    if graphs is not None:
        vertex_offsets, row_ptr, col, _ = concat_graphs(graphs)
    vo = np.ascontiguousarray(vertex_offsets, dtype=np.int32)
    rp_p, rp_kind, rp_keep, rp_len = _as_i32(row_ptr)
    c_p, c_kind, c_keep, m = _as_i32(col)
    if m > 0 and rp_kind != c_kind:
        raise ValueError("row_ptr and col must both be host or both be device arrays")
    h = ctypes.c_void_p(0)
    rc = lib().ktruss_load_batch(ctypes.byref(h), vo.shape[0] - 1, vo.ctypes.data, rp_len - 1, m,
                                 rp_p, c_p, rp_kind, _stream_ptr(stream))
    _check(rc, "ktruss_load_batch")
    return Graph(h.value, rp_len - 1, m)


class Server:
    """K-truss request server (ktruss_server_*): continuous batching of
    requests with different graphs and K.  submit() queues a host CSR;
    step() admits what fits, runs one batched peel round and returns the
    requests completed by it as (ticket, rounds, mask, support)."""

    def __init__(self, max_vertices: int, max_edges: int, max_requests: int = 256,
                 request_bytes: int | None = None, stream=None):
        if request_bytes is None:
            request_bytes = 12 * max_edges + 8 * max_vertices + 1024 * max_requests
        h = ctypes.c_void_p(0)
        rc = lib().ktruss_server_create(ctypes.byref(h), max_vertices, max_edges, max_requests,
                                        request_bytes, _stream_ptr(stream))
        _check(rc, "ktruss_server_create")
        self._h = h
        self._pending = {}

    def set_update(self, mode: int):
        """KTRUSS_OPT_UPDATE for the server's rounds (UPDATE_*)."""
        _check(lib().ktruss_server_set_option(self._h, OPT_UPDATE, mode),
               "ktruss_server_set_option")

    def set_reorder(self, on: bool):
        """KTRUSS_OPT_REORDER: requests relabelled by ascending degree at
        admission (True, default) or appended in their own numbering."""
        _check(lib().ktruss_server_set_option(self._h, OPT_REORDER, 1 if on else 0),
               "ktruss_server_set_option")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ktruss_server_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, row_ptr, col, K: int, support: bool = True, mask_out=None,
               support_out=None) -> int:
        """Queues one request.  mask_out / support_out: caller-owned host
        arrays (uint8 / int32, at least m entries, C-contiguous) that receive
        the outputs; allocated here when None."""
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        c = np.ascontiguousarray(col, dtype=np.int32)
        m = c.shape[0]

        def out(a, dtype):
            if a is None:
                return np.zeros(max(m, 1), dtype=dtype)
            if (not isinstance(a, np.ndarray) or a.dtype != dtype or a.ndim != 1
                    or a.shape[0] < m or not a.flags.c_contiguous):
                raise ValueError(f"output array must be C-contiguous {np.dtype(dtype).name}[>= {m}]")
            return a

        mask = out(mask_out, np.uint8)
        sup = out(support_out, np.int32) if support else None
        t = ctypes.c_int64(0)
        rc = lib().ktruss_server_submit(self._h, rp.shape[0] - 1, m, rp.ctypes.data,
                                        c.ctypes.data if m else None, K, mask.ctypes.data,
                                        sup.ctypes.data if sup is not None else None,
                                        ctypes.byref(t))
        _check(rc, "ktruss_server_submit")
        self._pending[t.value] = (mask[:m], sup[:m] if sup is not None else None)
        return t.value

    def step(self):
        nd = ctypes.c_int32(0)
        _check(lib().ktruss_server_step(self._h, ctypes.byref(nd)), "ktruss_server_step")
        out = []
        if nd.value:
            tk = np.zeros(nd.value, dtype=np.int64)
            rd = np.zeros(nd.value, dtype=np.int32)
            cnt = ctypes.c_int32(0)
            _check(lib().ktruss_server_take_done(self._h, tk.ctypes.data, rd.ctypes.data,
                                                 nd.value, ctypes.byref(cnt)),
                   "ktruss_server_take_done")
            for t, r in zip(tk[:cnt.value], rd[:cnt.value]):
                mask, sup = self._pending.pop(int(t))
                out.append((int(t), int(r), mask, sup))
        return out

    def status(self):
        q, a, e = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int64(0)
        _check(lib().ktruss_server_status(self._h, ctypes.byref(q), ctypes.byref(a),
                                          ctypes.byref(e)), "ktruss_server_status")
        return q.value, a.value, e.value


def serve_poisson(server, requests, rate, seed=0, clock=None, outputs=None, step_times=None):
    """Feeds (csr, K) requests to a Server with Poisson arrivals of the given
    rate (requests/s; None = all at time 0) in real time and steps it until
    every request is done.  outputs: optional (mask, support) host arrays per
    request (Server.submit's mask_out / support_out).  step_times: optional
    list that receives the host time (s) of every Server.step call.  Returns
    per-request latencies (s, arrival to completion), the makespan and the
    results by request index."""
    import time
    clock = clock or time.perf_counter
    rng = np.random.default_rng(seed)
    N = len(requests)
    arrivals = (np.zeros(N) if rate is None
                else np.cumsum(rng.exponential(1.0 / rate, size=N)))
    t0 = clock()
    i = 0
    ticket_of = {}
    latency = np.zeros(N)
    results = [None] * N
    done = 0
    while done < N:
        now = clock() - t0
        while i < N and arrivals[i] <= now:
            g, K = requests[i]
            mo, so = outputs[i] if outputs is not None else (None, None)
            ticket_of[server.submit(g.row_ptr, g.col, K, mask_out=mo, support_out=so)] = i
            i += 1
        q, a, _ = server.status()
        if q == 0 and a == 0:
            if i < N:
                time.sleep(max(0.0, min(0.001, arrivals[i] - (clock() - t0))))
            continue
        ts = clock()
        finished = server.step()
        if step_times is not None:
            step_times.append(clock() - ts)
        for t, r, mask, sup in finished:
            k = ticket_of.pop(t)
            latency[k] = (clock() - t0) - arrivals[k]
            results[k] = (r, mask, sup)
            done += 1
    return latency, clock() - t0, results


def trim_cache():
    """ktruss_trim_cache: frees the device blocks that freed handles left in
    the library's cache."""
    _check(lib().ktruss_trim_cache(), "ktruss_trim_cache")


NOALLOC_MAX_VERTICES = 1 << 19
NOALLOC_MAX_EDGES = 1 << 19


def support_noalloc(row_ptr, col, support_out=None, stream=None):
    """ktruss_support_noalloc: support of every edge of a device-resident CSR,
    computed by the library without allocating (its working memory is a fixed
    32 MiB array inside the library).  For callers that may not allocate on
    their path.  row_ptr/col: int32 cuda tensors; support_out: an int32 cuda
    tensor of m entries (allocated here when None, which the caller can avoid
    by passing one).  Returns (support_out, triangles)."""
    torch = _torch()
    n = row_ptr.shape[0] - 1
    m = col.shape[0]
    if support_out is None:
        support_out = torch.empty(max(m, 1), dtype=torch.int32, device=row_ptr.device)[:m]
    tri = ctypes.c_int64(0)
    rc = lib().ktruss_support_noalloc(n, m, row_ptr.data_ptr(), col.data_ptr() if m else None,
                                      support_out.data_ptr() if m else None,
                                      ctypes.addressof(tri), _stream_ptr(stream))
    _check(rc, "ktruss_support_noalloc")
    return support_out, tri.value


def ktruss(row_ptr, col, K: int, kernel: int = KERNEL_AUTO):
    """One-shot helper: load, run on the device, return (mask, support, stats)."""
    g = load(row_ptr, col)
    g.set_kernel(kernel)
    mask, sup = g.run(K)
    st = g.stats()
    g.close()
    return mask, sup, st
