"""Host-side checks of the C ABI: the library loads, exports every entry point
declared in include/jzt.h, and rejects bad arguments synchronously (no GPU
needed: these calls return before any CUDA work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    import __graft_entry__
    __graft_entry__._builder().build()
    import paper_2604_05885_gb300 as jzt
    return jzt


def test_exports_every_declared_symbol():
    jzt = _lib()
    hdr = open(os.path.join(ROOT, "include", "jzt.h")).read()
    declared = set(re.findall(r"\b(jzt_[a-z_]+)\s*\(", hdr))
    assert declared, "no declarations parsed"
    assert declared == set(jzt.SYMBOLS), declared ^ set(jzt.SYMBOLS)
    raw = ctypes.CDLL(jzt.LIB_PATH)
    for name in declared:
        assert hasattr(raw, name), name


def test_version():
    jzt = _lib()
    assert "sm_103a" in jzt.version()


def test_workspace_bytes_grows_and_validates():
    jzt = _lib()
    a = jzt.workspace_bytes(1000)
    b = jzt.workspace_bytes(1 << 20)
    c = jzt.workspace_bytes(1 << 27, 16)
    assert 0 < a < b < c
    assert c < 40 * (1 << 30)  # stays well inside HBM at 2^27 points
    for bad in (0, -5, 1 << 31):
        with pytest.raises(jzt.JztError) as e:
            jzt.workspace_bytes(bad)
        assert e.value.code == jzt.JZT_ERR_INVALID
    assert jzt.workspace_bytes(1000, 256) > jzt.workspace_bytes(1000, 32)
    with pytest.raises(jzt.JztError):
        jzt.workspace_bytes(100, 257)
    # the key sort's choice changes no workspace part
    assert jzt.workspace_bytes(1 << 20, 16, {"lsd_sort": 1}) == jzt.workspace_bytes(1 << 20, 16)
    for p in ({"nmax0": 33}, {"nmax0": -1}, {"plane_factor": 1}, {"heap_size": 17},
              {"alloc_fac_ilist": -1.0}, {"lsd_sort": 2}, {"lsd_sort": -1}):
        with pytest.raises(jzt.JztError) as e:
            jzt.workspace_bytes(1000, 0, p)
        assert e.value.code == jzt.JZT_ERR_INVALID
    p = jzt.Params()
    p.reserved[0] = 1
    with pytest.raises(jzt.JztError):
        jzt.workspace_bytes(1000, 0, p)


def test_synchronous_argument_errors():
    jzt = _lib()
    lib = jzt.lib
    vp = ctypes.c_void_p
    h = vp(0)
    # null pointers / bad N / misaligned workspace: rejected before any CUDA call
    assert lib.jzt_build(None, 10, 0.0, None, vp(256), 1 << 20, None, ctypes.byref(h)) == jzt.JZT_ERR_INVALID
    assert lib.jzt_build(vp(256), 0, 0.0, None, vp(256), 1 << 20, None, ctypes.byref(h)) == jzt.JZT_ERR_INVALID
    assert lib.jzt_build(vp(256), 10, 0.0, None, vp(260), 1 << 20, None, ctypes.byref(h)) == jzt.JZT_ERR_INVALID
    assert lib.jzt_build(vp(258), 10, 0.0, None, vp(256), 1 << 20, None, ctypes.byref(h)) == jzt.JZT_ERR_INVALID
    assert lib.jzt_build(vp(256), 10, float("nan"), None, vp(256), 1 << 20, None,
                         ctypes.byref(h)) == jzt.JZT_ERR_INVALID
    assert lib.jzt_build(vp(256), 10, 0.0, None, vp(256), 16, None, ctypes.byref(h)) == jzt.JZT_ERR_WORKSPACE
    assert b"workspace too small" in lib.jzt_last_error()
    assert lib.jzt_tree_knn(None, 4, 0, vp(256), vp(256), None) == jzt.JZT_ERR_INVALID
    assert lib.jzt_tree_fof(None, 0.1, vp(256), None) == jzt.JZT_ERR_INVALID
    assert lib.jzt_knn(vp(256), 1000, 257, 0.0, vp(256), vp(256), vp(256), 1 << 20, None) == jzt.JZT_ERR_UNSUPPORTED
    assert lib.jzt_knn(vp(256), 10, 11, 0.0, vp(256), vp(256), vp(256), 1 << 20, None) == jzt.JZT_ERR_INVALID
    assert lib.jzt_knn(vp(256), 10, 0, 0.0, vp(256), vp(256), vp(256), 1 << 20, None) == jzt.JZT_ERR_INVALID
    assert lib.jzt_fof(vp(256), 10, 0.0, 0.0, vp(256), vp(256), 1 << 20, None) == jzt.JZT_ERR_INVALID
    assert lib.jzt_fof(vp(256), 10, 0.6, 1.0, vp(256), vp(256), 1 << 20, None) == jzt.JZT_ERR_INVALID
    assert lib.jzt_fof(vp(256), 10, float("inf"), 0.0, vp(256), vp(256), 1 << 20, None) == jzt.JZT_ERR_INVALID
    assert lib.jzt_status(None, None, None) == jzt.JZT_ERR_INVALID
    assert lib.jzt_tree_arrays(None, None, None, None) == jzt.JZT_ERR_INVALID
    lib.jzt_tree_free(None)


def test_product_has_no_oracle_dependency():
    """The CUDA path never imports, links or runs the oracle."""
    pkg = os.path.join(ROOT, "paper_2604_05885_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.lower().replace("oracle-free", ""), f


def test_batch_queue_scratch_and_job_checks():
    """jzt_batch_queue_bytes is host arithmetic; jzt_batch_run_queue and
    jzt_batch_run refuse bad jobs before any CUDA work (per-job leaf capacity
    out of range, missing scratch)."""
    jzt = _lib()
    sz = [ctypes.c_size_t(0) for _ in range(3)]
    for n, b in zip((0, 10, 1000), sz):
        assert jzt.lib.jzt_batch_queue_bytes(n, ctypes.byref(b)) == 0
    assert 0 < sz[0].value < sz[1].value < sz[2].value
    assert sz[2].value % 256 == 0
    assert jzt.lib.jzt_batch_queue_bytes(-1, ctypes.byref(sz[0])) == jzt.JZT_ERR_INVALID
    jobs = (jzt.Job * 1)()
    J = jobs[0]
    J.d_xyz, J.n, J.op, J.k, J.lane, J.nmax0 = 0x1000, 100, jzt.JZT_OP_KNN, 8, 0, 33
    J.d_idx, J.d_dist2 = 0x2000, 0x3000
    ws = (ctypes.c_void_p * 1)(0x100000)
    wsb = (ctypes.c_size_t * 1)(1 << 30)
    streams = (ctypes.c_void_p * 1)(None)
    rc = jzt.lib.jzt_batch_run(jobs, 1, None, ws, wsb, streams, 1, None, ctypes.c_void_p(0x4000))
    assert rc == jzt.JZT_ERR_INVALID and b"nmax0" in jzt.lib.jzt_last_error()
    rc = jzt.lib.jzt_batch_run_queue(jobs, 1, None, ws, wsb, streams, 1, None, None, 0, ctypes.c_void_p(0x4000))
    assert rc == jzt.JZT_ERR_WORKSPACE
