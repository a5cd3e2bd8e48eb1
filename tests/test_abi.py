"""The C ABI library builds for sm_103a, loads, and exports every function
declared in include/ktruss.h (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

import paper_2009_07929_gb300 as kt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ktruss.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ktruss_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("ktruss_load_csr", "ktruss_run", "ktruss_stats", "ktruss_free", "ktruss_strerror"):
        assert f in names


def test_library_exports_every_declared_symbol():
    L = kt.lib()
    for name in declared_functions():
        assert hasattr(L, name), name


def test_error_strings_and_version_without_gpu():
    L = kt.lib()
    assert L.ktruss_version() >= 100
    for code in (kt.OK, kt.EINVAL, kt.ENOMEM, kt.ECUDA, kt.ETIMEOUT, kt.EBUSY):
        assert L.ktruss_strerror(code)
    assert L.ktruss_strerror(-99) == b"unknown error"


def test_argument_checks_before_any_cuda_call():
    L = kt.lib()
    h = ctypes.c_void_p(0)
    # NULL out-pointer, negative sizes, NULL arrays and bad kinds are rejected on the host
    assert L.ktruss_load_csr(None, 1, 0, None, None, kt.HOST, None) == kt.EINVAL
    assert L.ktruss_load_csr(ctypes.byref(h), -1, 0, None, None, kt.HOST, None) == kt.EINVAL
    assert L.ktruss_load_csr(ctypes.byref(h), 3, -1, None, None, kt.HOST, None) == kt.EINVAL
    assert L.ktruss_load_csr(ctypes.byref(h), 3, 1 << 31, None, None, kt.HOST, None) == kt.EINVAL
    rp = (ctypes.c_int32 * 2)(0, 0)
    assert L.ktruss_load_csr(ctypes.byref(h), 1, 0, rp, None, 7, None) == kt.EINVAL
    assert L.ktruss_run(None, 3, None, None, kt.DEVICE, None) == kt.EINVAL
    assert L.ktruss_stats(None, None) == kt.EINVAL
    assert L.ktruss_set_option(None, kt.OPT_TIMING, 1) == kt.EINVAL
    assert L.ktruss_set_option(None, kt.OPT_LIGHT_MERGE, 64) == kt.EINVAL
    assert L.ktruss_autotune(None, None, 1, 1, None, None) == kt.EINVAL
    assert L.ktruss_server_set_option(None, kt.OPT_UPDATE, 2) == kt.EINVAL
    assert L.ktruss_decompose(None, None, None, kt.DEVICE, None) == kt.EINVAL
    assert L.ktruss_trim_cache() == kt.OK  # empty cache: no CUDA call
    L.ktruss_free(None)


def test_batch_server_and_noalloc_argument_checks_without_gpu():
    """Malformed arguments of the batch, server and allocation-free entry
    points are rejected on the host, before any CUDA call."""
    L = kt.lib()
    h = ctypes.c_void_p(0)
    rp = (ctypes.c_int32 * 5)(0, 0, 0, 0, 0)

    def vo(*v):
        return (ctypes.c_int32 * len(v))(*v)

    # batches: out-pointer, graph count, vertex offsets (start 0, end n, monotone)
    assert L.ktruss_load_batch(None, 1, vo(0, 4), 4, 0, rp, None, kt.HOST, None) == kt.EINVAL
    assert L.ktruss_load_batch(ctypes.byref(h), 0, vo(0), 4, 0, rp, None, kt.HOST, None) == kt.EINVAL
    assert L.ktruss_load_batch(ctypes.byref(h), 1, None, 4, 0, rp, None, kt.HOST, None) == kt.EINVAL
    assert L.ktruss_load_batch(ctypes.byref(h), 1, vo(1, 4), 4, 0, rp, None, kt.HOST,
                               None) == kt.EINVAL
    assert L.ktruss_load_batch(ctypes.byref(h), 1, vo(0, 3), 4, 0, rp, None, kt.HOST,
                               None) == kt.EINVAL
    assert L.ktruss_load_batch(ctypes.byref(h), 2, vo(0, 3, 2), 2, 0, rp, None, kt.HOST,
                               None) == kt.EINVAL
    assert L.ktruss_load_batch(ctypes.byref(h), 2, vo(0, 2, 4), 4, 0, rp, None, 9,
                               None) == kt.EINVAL
    assert not h.value
    G = ctypes.c_int32(0)
    n, m = ctypes.c_int32(0), ctypes.c_int64(0)
    assert L.ktruss_batch_size(None, ctypes.byref(G)) == kt.EINVAL
    assert L.ktruss_run_batch(None, None, None, None, None, kt.DEVICE, None) == kt.EINVAL
    assert L.ktruss_graph_size(None, ctypes.byref(n), ctypes.byref(m)) == kt.EINVAL
    # server: sizes and budget at creation; every call needs a server
    srv = ctypes.c_void_p(0)
    assert L.ktruss_server_create(None, 16, 16, 4, 0, None) == kt.EINVAL
    assert L.ktruss_server_create(ctypes.byref(srv), 0, 16, 4, 0, None) == kt.EINVAL
    assert L.ktruss_server_create(ctypes.byref(srv), 16, 0, 4, 0, None) == kt.EINVAL
    assert L.ktruss_server_create(ctypes.byref(srv), 16, 1 << 31, 4, 0, None) == kt.EINVAL
    assert L.ktruss_server_create(ctypes.byref(srv), 16, 16, 0, 0, None) == kt.EINVAL
    assert L.ktruss_server_create(ctypes.byref(srv), 16, 16, 4, -1, None) == kt.EINVAL
    assert not srv.value
    t = ctypes.c_int64(0)
    nd, q, a = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    e = ctypes.c_int64(0)
    assert L.ktruss_server_submit(None, 1, 0, rp, None, 3, None, None, ctypes.byref(t)) == kt.EINVAL
    assert L.ktruss_server_step(None, ctypes.byref(nd)) == kt.EINVAL
    assert L.ktruss_server_take_done(None, None, None, 0, ctypes.byref(nd)) == kt.EINVAL
    assert L.ktruss_server_status(None, ctypes.byref(q), ctypes.byref(a),
                                  ctypes.byref(e)) == kt.EINVAL
    L.ktruss_server_free(None)
    # allocation-free supports: sizes above the fixed scratch's limits, NULL arrays
    assert L.ktruss_support_noalloc(kt.NOALLOC_MAX_VERTICES + 1, 0, rp, None, None, None,
                                    None) == kt.EINVAL
    assert L.ktruss_support_noalloc(4, kt.NOALLOC_MAX_EDGES + 1, rp, rp, rp, None,
                                    None) == kt.EINVAL
    assert L.ktruss_support_noalloc(-1, 0, rp, None, None, None, None) == kt.EINVAL
    assert L.ktruss_support_noalloc(4, 2, None, rp, rp, None, None) == kt.EINVAL
    assert L.ktruss_support_noalloc(4, 2, rp, None, rp, None, None) == kt.EINVAL
    assert L.ktruss_support_noalloc(4, 2, rp, rp, None, None, None) == kt.EINVAL


def test_build_is_for_sm_103a():
    from paper_2009_07929_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)
    assert os.path.exists(kt.library_path())
