"""Python binding of libjzt.so: exact kNN and FoF on GB300 (sm_103a).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libjzt.so behind the C ABI declared in include/jzt.h.  PyTorch
provides device memory (workspace and outputs) and the current stream.

The functions mirror the C entry points:

* ``workspace_bytes(n, k=0, params=None)``
* ``build(xyz, periodic_L=0.0, params=None, workspace=None) -> Tree``
* ``Tree.knn(k, order=0) -> (idx int32 [N,k], dist2 float32 [N,k])``
* ``Tree.fof(b) -> labels int32 [N]``
* ``knn(xyz, k, periodic_L=0.0)`` / ``fof(xyz, b, periodic_L=0.0)`` one-call forms
* ``status(workspace) -> dict``

A missing or unloadable library raises at import time: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libjzt.so")

JZT_OK = 0
JZT_ERR_INVALID = -1
JZT_ERR_UNSUPPORTED = -2
JZT_ERR_CUDA = -3
JZT_ERR_WORKSPACE = -4
JZT_ERR_CAPACITY = -5
JZT_ERR_INPUT = -6
JZT_ERR_TIMEOUT = -7
JZT_ERR_INTERNAL = -8
_NAMES = {0: "ok", -1: "invalid", -2: "unsupported", -3: "cuda", -4: "workspace",
          -5: "capacity", -6: "input", -7: "timeout", -8: "internal"}

# Every entry point declared in include/jzt.h.
SYMBOLS = ("jzt_workspace_bytes", "jzt_build", "jzt_tree_knn", "jzt_tree_fof", "jzt_knn", "jzt_fof",
           "jzt_status", "jzt_tree_arrays", "jzt_tree_plane", "jzt_tree_free", "jzt_last_error",
           "jzt_version", "jzt_profile_enable", "jzt_profile_read", "jzt_profile_phase_name",
           "jzt_knn_noalloc", "jzt_batch_run", "jzt_workspace_bytes_query", "jzt_build_query",
           "jzt_knn_query", "jzt_tree_fof_catalogue", "jzt_selftest_wait", "jzt_batch_queue_bytes",
           "jzt_batch_run_queue")
JZT_OP_KNN = 0
JZT_OP_FOF = 1


class JztError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    """Mirror of jzt_params (zero fields take the library defaults)."""
    _fields_ = [("nmax0", ctypes.c_int32), ("plane_factor", ctypes.c_int32),
                ("n_target", ctypes.c_int32), ("ngr", ctypes.c_int32),
                ("alloc_fac_nodes", ctypes.c_float), ("alloc_fac_ilist", ctypes.c_float),
                ("heap_size", ctypes.c_int32), ("reg_fmax", ctypes.c_float), ("float_order", ctypes.c_int32),
                ("lsd_sort", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class Job(ctypes.Structure):
    """Mirror of jzt_job."""
    _fields_ = [("d_xyz", ctypes.c_void_p), ("n", ctypes.c_int64), ("periodic_L", ctypes.c_float),
                ("op", ctypes.c_int32), ("k", ctypes.c_int32), ("b", ctypes.c_float), ("lane", ctypes.c_int32),
                ("nmax0", ctypes.c_int32), ("d_idx", ctypes.c_void_p), ("d_dist2", ctypes.c_void_p),
                ("d_labels", ctypes.c_void_p)]


class StatusInfo(ctypes.Structure):
    _fields_ = [("code", ctypes.c_int32), ("detail", ctypes.c_int32),
                ("required_bytes", ctypes.c_int64), ("ilist_entries", ctypes.c_int64),
                ("n_planes", ctypes.c_int32), ("sort_path", ctypes.c_int32),
                ("n_nodes", ctypes.c_int64 * 16), ("knn_pairs", ctypes.c_int64),
                ("fof_pairs", ctypes.c_int64), ("knn_stats", ctypes.c_int64 * 8),
                ("knn_plane_entries", ctypes.c_int64 * 16)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, f32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_size_t
    lib.jzt_workspace_bytes.argtypes = [i64, ctypes.c_int, ctypes.POINTER(Params), ctypes.POINTER(sz)]
    lib.jzt_build.argtypes = [vp, i64, f32, ctypes.POINTER(Params), vp, sz, vp, ctypes.POINTER(vp)]
    lib.jzt_tree_knn.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp]
    lib.jzt_tree_fof.argtypes = [vp, f32, vp, vp]
    lib.jzt_knn.argtypes = [vp, i64, ctypes.c_int, f32, vp, vp, vp, sz, vp]
    lib.jzt_fof.argtypes = [vp, i64, f32, f32, vp, vp, sz, vp]
    lib.jzt_status.argtypes = [vp, vp, ctypes.POINTER(StatusInfo)]
    lib.jzt_tree_arrays.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i32)]
    lib.jzt_tree_plane.argtypes = [vp, ctypes.c_int, i64, ctypes.POINTER(i64), vp, vp, vp, vp]
    lib.jzt_profile_enable.argtypes = [ctypes.c_int]
    lib.jzt_profile_enable.restype = ctypes.c_int
    lib.jzt_profile_read.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64), ctypes.c_int,
                                     ctypes.POINTER(i64)]
    lib.jzt_profile_read.restype = ctypes.c_int
    lib.jzt_profile_phase_name.argtypes = [ctypes.c_int]
    lib.jzt_profile_phase_name.restype = ctypes.c_char_p
    lib.jzt_knn_noalloc.argtypes = [vp, i64, ctypes.c_int, f32, vp, vp, vp, ctypes.POINTER(StatusInfo)]
    lib.jzt_knn_noalloc.restype = ctypes.c_int
    lib.jzt_batch_run.argtypes = [ctypes.POINTER(Job), ctypes.c_int, ctypes.POINTER(Params),
                                  ctypes.POINTER(vp), ctypes.POINTER(sz), ctypes.POINTER(vp), ctypes.c_int, vp, vp]
    lib.jzt_batch_run.restype = ctypes.c_int
    lib.jzt_batch_queue_bytes.argtypes = [ctypes.c_int, ctypes.POINTER(sz)]
    lib.jzt_batch_queue_bytes.restype = ctypes.c_int
    lib.jzt_batch_run_queue.argtypes = [ctypes.POINTER(Job), ctypes.c_int, ctypes.POINTER(Params),
                                        ctypes.POINTER(vp), ctypes.POINTER(sz), ctypes.POINTER(vp), ctypes.c_int, vp,
                                        vp, sz, vp]
    lib.jzt_batch_run_queue.restype = ctypes.c_int
    lib.jzt_workspace_bytes_query.argtypes = [i64, i64, ctypes.c_int, ctypes.POINTER(Params), ctypes.POINTER(sz)]
    lib.jzt_build_query.argtypes = [vp, i64, vp, i64, f32, ctypes.POINTER(Params), vp, sz, vp, ctypes.POINTER(vp)]
    lib.jzt_knn_query.argtypes = [vp, i64, vp, i64, ctypes.c_int, f32, vp, vp, vp, sz, vp]
    lib.jzt_tree_fof_catalogue.argtypes = [vp, f32, vp, ctypes.c_int, f32, vp, vp, vp, i64, vp, vp]
    lib.jzt_selftest_wait.argtypes = [ctypes.c_int, ctypes.c_longlong, vp, sz, vp, ctypes.POINTER(StatusInfo)]
    lib.jzt_selftest_wait.restype = ctypes.c_int
    for name in ("jzt_workspace_bytes_query", "jzt_build_query", "jzt_knn_query", "jzt_tree_fof_catalogue"):
        getattr(lib, name).restype = ctypes.c_int
    lib.jzt_tree_free.argtypes = [vp]
    lib.jzt_tree_free.restype = None
    lib.jzt_last_error.restype = ctypes.c_char_p
    lib.jzt_version.restype = ctypes.c_char_p
    for name in ("jzt_workspace_bytes", "jzt_build", "jzt_tree_knn", "jzt_tree_fof", "jzt_knn",
                 "jzt_fof", "jzt_status", "jzt_tree_arrays", "jzt_tree_plane"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


lib = _load()


def version() -> str:
    return lib.jzt_version().decode()


def _check(rc: int):
    if rc != JZT_OK:
        raise JztError(rc, lib.jzt_last_error().decode())


def _params(params) -> ctypes.POINTER(Params) | None:
    if params is None:
        return None
    if isinstance(params, Params):
        return ctypes.pointer(params)
    p = Params()
    for k, v in dict(params).items():
        setattr(p, k, v)
    return ctypes.pointer(p)


def _stream(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def workspace_bytes(n: int, k: int = 0, params=None) -> int:
    out = ctypes.c_size_t(0)
    _check(lib.jzt_workspace_bytes(int(n), int(k), _params(params), ctypes.byref(out)))
    return int(out.value)


def alloc_workspace(n: int, k: int = 0, params=None, device=None) -> torch.Tensor:
    nb = workspace_bytes(n, k, params)
    return torch.empty(nb, dtype=torch.uint8, device=device or "cuda")


def _check_xyz(xyz: torch.Tensor):
    if not (isinstance(xyz, torch.Tensor) and xyz.is_cuda and xyz.dtype == torch.float32
            and xyz.dim() == 2 and xyz.shape[1] == 3 and xyz.is_contiguous()):
        raise ValueError("xyz must be a contiguous CUDA float32 tensor of shape (N, 3)")


def status(workspace: torch.Tensor, stream=None, raise_on_error: bool = False) -> dict:
    """Synchronise the stream and read the workspace status block."""
    info = StatusInfo()
    rc = lib.jzt_status(ctypes.c_void_p(workspace.data_ptr()), ctypes.c_void_p(_stream(stream)),
                        ctypes.byref(info))
    if rc == JZT_ERR_CUDA or rc == JZT_ERR_INVALID:
        _check(rc)
    out = dict(code=info.code, name=_NAMES.get(info.code, str(info.code)), detail=info.detail,
               required_bytes=info.required_bytes, ilist_entries=info.ilist_entries,
               n_planes=info.n_planes, sort_path=info.sort_path, n_nodes=[info.n_nodes[i] for i in range(16)],
               knn_pairs=info.knn_pairs, fof_pairs=info.fof_pairs,
               knn_stats=[info.knn_stats[i] for i in range(8)],
               knn_plane_entries=[info.knn_plane_entries[i] for i in range(16)])
    if raise_on_error and info.code != JZT_OK:
        raise JztError(info.code, lib.jzt_last_error().decode())
    return out


def phase_names() -> list[str]:
    out = []
    while True:
        nm = lib.jzt_profile_phase_name(len(out))
        if nm is None:
            return out
        out.append(nm.decode())


def profile_enable(on: bool = True):
    lib.jzt_profile_enable(1 if on else 0)


def profile_read() -> tuple[dict, dict, int]:
    """(ms per phase, instances per phase, kernel launches) since the last read."""
    names = phase_names()
    n = len(names)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    launches = ctypes.c_int64(0)
    _check(lib.jzt_profile_read(ms, cnt, n, ctypes.byref(launches)))
    return ({names[i]: ms[i] for i in range(n)}, {names[i]: cnt[i] for i in range(n)}, int(launches.value))


def _group_dtype():
    import numpy as np
    return np.dtype([("label", "<i4"), ("count", "<i4"), ("offset", "<i8"), ("mass", "<f4"),
                     ("x_cm", "<f4", (3,)), ("v_cm", "<f4", (3,)), ("r_inertia", "<f4")])


GROUP_DTYPE = _group_dtype()  # jzt_group, 48 bytes


class Tree:
    """A tree built in a caller-owned workspace (see jzt_build)."""

    def __init__(self, xyz: torch.Tensor, periodic_L: float = 0.0, params=None,
                 workspace: torch.Tensor | None = None, stream=None, k_max: int = 32):
        _check_xyz(xyz)
        n = xyz.shape[0]
        self.n = n
        self.n_rows = n
        self.periodic_L = float(periodic_L)
        self.params = params
        self.workspace = workspace if workspace is not None else alloc_workspace(
            n, min(int(k_max), n, 32), params, xyz.device)
        self._h = ctypes.c_void_p(0)
        _check(lib.jzt_build(ctypes.c_void_p(xyz.data_ptr()), n, self.periodic_L, _params(params),
                             ctypes.c_void_p(self.workspace.data_ptr()), self.workspace.numel(),
                             ctypes.c_void_p(_stream(stream)), ctypes.byref(self._h)))

    def knn(self, k: int, order: int = 0, out=None, stream=None):
        dev = self.workspace.device
        if out is None:
            idx = torch.empty((self.n_rows, k), dtype=torch.int32, device=dev)
            d2 = torch.empty((self.n_rows, k), dtype=torch.float32, device=dev)
        else:
            idx, d2 = out
        _check(lib.jzt_tree_knn(self._h, int(k), int(order), ctypes.c_void_p(idx.data_ptr()),
                                ctypes.c_void_p(d2.data_ptr()), ctypes.c_void_p(_stream(stream))))
        return idx, d2

    def fof(self, b: float, out=None, stream=None):
        lab = out if out is not None else torch.empty(self.n, dtype=torch.int32, device=self.workspace.device)
        _check(lib.jzt_tree_fof(self._h, float(b), ctypes.c_void_p(lab.data_ptr()),
                                ctypes.c_void_p(_stream(stream))))
        return lab

    def fof_catalogue(self, b: float, vel=None, min_count: int = 20, particle_mass: float = 1.0,
                      cap_groups: int | None = None, stream=None):
        """FoF labels plus the catalogue of groups with >= min_count points (jzt_tree_fof_catalogue).
        Returns (labels [N] int32, order [N] int32 original indices in group order,
        groups: host numpy structured array with GROUP_DTYPE fields, in group order)."""
        import numpy as np
        dev = self.workspace.device
        n = self.n
        cap = int(cap_groups) if cap_groups is not None else n // max(1, int(min_count)) + 1
        labels = torch.empty(n, dtype=torch.int32, device=dev)
        order = torch.empty(n, dtype=torch.int32, device=dev)
        gbuf = torch.empty(max(cap, 1) * GROUP_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        ng = torch.zeros(1, dtype=torch.int64, device=dev)
        if vel is not None:
            _check_xyz(vel)
        _check(lib.jzt_tree_fof_catalogue(self._h, float(b), ctypes.c_void_p(vel.data_ptr() if vel is not None else 0),
                                          int(min_count), float(particle_mass), ctypes.c_void_p(labels.data_ptr()),
                                          ctypes.c_void_p(order.data_ptr()), ctypes.c_void_p(gbuf.data_ptr()), cap,
                                          ctypes.c_void_p(ng.data_ptr()), ctypes.c_void_p(_stream(stream))))
        self.status(stream, raise_on_error=True)
        k = min(int(ng.item()), cap)
        groups = np.frombuffer(gbuf[:k * GROUP_DTYPE.itemsize].cpu().numpy().tobytes(), dtype=GROUP_DTYPE)
        return labels, order, groups

    def arrays(self):
        """(sorted keys uint64 view as int64 [N] -- None for the float z-order, which
        has no keys --, sorted points float32 [N,4], n_planes)."""
        kp, pp, npl = ctypes.c_void_p(0), ctypes.c_void_p(0), ctypes.c_int32(0)
        _check(lib.jzt_tree_arrays(self._h, ctypes.byref(kp), ctypes.byref(pp), ctypes.byref(npl)))
        ws = self.workspace
        base = ws.data_ptr()
        poff = pp.value - base
        keys = None
        if kp.value:
            koff = kp.value - base
            keys = ws[koff:koff + 8 * self.n].view(torch.int64)
        pts = ws[poff:poff + 16 * self.n].view(torch.float32).view(self.n, 4)
        return keys, pts, int(npl.value)

    def plane(self, p: int, stream=None):
        """Host copies of plane p: (spl int32 [n+1], count int32 [n], box float32 [n,6])."""
        import numpy as np
        nn = ctypes.c_int64(0)
        _check(lib.jzt_tree_plane(self._h, int(p), 0, ctypes.byref(nn), None, None, None,
                                  ctypes.c_void_p(_stream(stream))))
        n = int(nn.value)
        spl = np.empty(n + 1, np.int32)
        cnt = np.empty(max(n, 1), np.int32)
        box = np.empty((max(n, 1), 6), np.float32)
        _check(lib.jzt_tree_plane(self._h, int(p), n, ctypes.byref(nn),
                                  ctypes.c_void_p(spl.ctypes.data), ctypes.c_void_p(cnt.ctypes.data),
                                  ctypes.c_void_p(box.ctypes.data), ctypes.c_void_p(_stream(stream))))
        return spl, cnt[:n], box[:n]

    def status(self, stream=None, raise_on_error: bool = False) -> dict:
        return status(self.workspace, stream, raise_on_error)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib.jzt_tree_free(h)
            self._h = ctypes.c_void_p(0)


def workspace_bytes_query(n_src: int, n_qry: int, k: int = 0, params=None) -> int:
    out = ctypes.c_size_t(0)
    _check(lib.jzt_workspace_bytes_query(int(n_src), int(n_qry), int(k), _params(params), ctypes.byref(out)))
    return int(out.value)


class QueryTree(Tree):
    """A tree over source points and separate query points (jzt_build_query):
    knn(k) returns one row per query point listing source indices."""

    def __init__(self, src: torch.Tensor, qry: torch.Tensor, periodic_L: float = 0.0, params=None,
                 workspace: torch.Tensor | None = None, stream=None, k_max: int = 32):
        _check_xyz(src)
        _check_xyz(qry)
        self.n = src.shape[0] + qry.shape[0]
        self.n_src = src.shape[0]
        self.n_rows = qry.shape[0]
        self.periodic_L = float(periodic_L)
        self.params = params
        self.workspace = workspace if workspace is not None else torch.empty(
            workspace_bytes_query(self.n_src, self.n_rows, min(int(k_max), self.n_src, 256), params),
            dtype=torch.uint8, device=src.device)
        self._h = ctypes.c_void_p(0)
        _check(lib.jzt_build_query(ctypes.c_void_p(src.data_ptr()), self.n_src, ctypes.c_void_p(qry.data_ptr()),
                                   self.n_rows, self.periodic_L, _params(params),
                                   ctypes.c_void_p(self.workspace.data_ptr()), self.workspace.numel(),
                                   ctypes.c_void_p(_stream(stream)), ctypes.byref(self._h)))


def build_query(src, qry, periodic_L=0.0, params=None, workspace=None, stream=None, k_max=32) -> QueryTree:
    return QueryTree(src, qry, periodic_L, params, workspace, stream, k_max)


def knn_query(src: torch.Tensor, qry: torch.Tensor, k: int, periodic_L: float = 0.0, workspace=None, stream=None,
              check=True):
    """One-call kNN of query points among source points (jzt_knn_query); returns
    (idx [N_qry, k] int32 source indices, dist2 [N_qry, k] float32)."""
    _check_xyz(src)
    _check_xyz(qry)
    ns, nq = src.shape[0], qry.shape[0]
    ws = workspace if workspace is not None else torch.empty(workspace_bytes_query(ns, nq, min(k, ns)),
                                                             dtype=torch.uint8, device=src.device)
    idx = torch.empty((nq, k), dtype=torch.int32, device=src.device)
    d2 = torch.empty((nq, k), dtype=torch.float32, device=src.device)
    _check(lib.jzt_knn_query(ctypes.c_void_p(src.data_ptr()), ns, ctypes.c_void_p(qry.data_ptr()), nq, int(k),
                             float(periodic_L), ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(d2.data_ptr()),
                             ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(_stream(stream))))
    if check:
        status(ws, stream, raise_on_error=True)
    return idx, d2


def build(xyz, periodic_L=0.0, params=None, workspace=None, stream=None, k_max=32) -> Tree:
    return Tree(xyz, periodic_L, params, workspace, stream, k_max)


def knn(xyz: torch.Tensor, k: int, periodic_L: float = 0.0, workspace=None, stream=None, check=True, out=None):
    """One-call exact kNN (jzt_knn); returns (idx [N,k] int32, dist2 [N,k] float32)."""
    _check_xyz(xyz)
    n = xyz.shape[0]
    ws = workspace if workspace is not None else alloc_workspace(n, min(k, n), None, xyz.device)
    if out is None:
        idx = torch.empty((n, k), dtype=torch.int32, device=xyz.device)
        d2 = torch.empty((n, k), dtype=torch.float32, device=xyz.device)
    else:
        idx, d2 = out
    _check(lib.jzt_knn(ctypes.c_void_p(xyz.data_ptr()), n, int(k), float(periodic_L),
                       ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(d2.data_ptr()),
                       ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(_stream(stream))))
    if check:
        status(ws, stream, raise_on_error=True)
    return idx, d2


def fof(xyz: torch.Tensor, b: float, periodic_L: float = 0.0, workspace=None, stream=None, check=True, out=None):
    """One-call FoF (jzt_fof); returns labels [N] int32 (smallest index of each group)."""
    _check_xyz(xyz)
    n = xyz.shape[0]
    ws = workspace if workspace is not None else alloc_workspace(n, 0, None, xyz.device)
    lab = out if out is not None else torch.empty(n, dtype=torch.int32, device=xyz.device)
    _check(lib.jzt_fof(ctypes.c_void_p(xyz.data_ptr()), n, float(b), float(periodic_L),
                       ctypes.c_void_p(lab.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                       ctypes.c_void_p(_stream(stream))))
    if check:
        status(ws, stream, raise_on_error=True)
    return lab


def assign_lanes(sizes, n_lanes: int) -> list[int]:
    """Lane of every job: longest processing time first, each job to the lane
    with the fewest points so far (the lowest lane on ties).  Host logic only."""
    order = sorted(range(len(sizes)), key=lambda j: -sizes[j])
    load = [0] * n_lanes
    lane_of = [0] * len(sizes)
    for j in order:
        lane = min(range(n_lanes), key=lambda q: load[q])
        lane_of[j] = lane
        load[lane] += sizes[j]
    return lane_of


class Batch:
    """Independent kNN / FoF jobs run on concurrent lanes through jzt_batch_run,
    optionally captured once into a CUDA graph and replayed.

    sets: list of dicts with keys ``points`` (contiguous CUDA float32 tensor N x 3),
    ``op`` ('knn' or 'fof'), ``k`` (kNN), ``b`` (FoF), ``periodic_L`` (default 0).
    Jobs are spread over ``n_lanes`` lanes by longest-processing-time order (each
    to the least loaded lane); every lane gets one workspace sized for its largest
    job.  Outputs: ``outputs[j]`` is (idx, dist2) for kNN jobs and labels for FoF.

    queue=True runs the batch through jzt_batch_run_queue instead: one workspace
    per job, and the kNN LeafToLeaf of all jobs (k <= 32) in persistent launches
    over a device work queue (same results).

    nmax0_of: optional callable N -> leaf capacity N_max^(0) (1..32, 0 = params')
    giving each job its own leaf capacity by its size (see autotune.tune).
    """

    def __init__(self, sets, n_lanes: int = 8, params=None, graph: bool = True, device=None, queue: bool = False,
                 nmax0_of=None):
        if not sets:
            raise ValueError("empty batch")
        dev = torch.device(device) if device is not None else sets[0]["points"].device
        self.sets = sets
        self.params = params
        nj = len(sets)
        n_lanes = max(1, min(int(n_lanes), nj))
        self.n_lanes = n_lanes
        sizes = [int(s["points"].shape[0]) for s in sets]
        lane_of = assign_lanes(sizes, n_lanes)
        self.queue = bool(queue)
        self.job_nmax0 = [int(nmax0_of(n)) if nmax0_of else 0 for n in sizes]
        need = [0] * n_lanes
        job_need = []
        for j, st in enumerate(sets):
            _check_xyz(st["points"])
            k = int(st.get("k", 0)) if st["op"] == "knn" else 0
            pj = dict(params or {})
            if self.job_nmax0[j]:
                pj["nmax0"] = self.job_nmax0[j]
            job_need.append(workspace_bytes(sizes[j], min(k, sizes[j]), pj or None))
            need[lane_of[j]] = max(need[lane_of[j]], job_need[-1])
        if self.queue:
            self.ws = [torch.empty(b, dtype=torch.uint8, device=dev) for b in job_need]
            qb = ctypes.c_size_t(0)
            _check(lib.jzt_batch_queue_bytes(nj, ctypes.byref(qb)))
            self.scratch = torch.empty(int(qb.value), dtype=torch.uint8, device=dev)
        else:
            self.ws = [torch.empty(need[q], dtype=torch.uint8, device=dev) for q in range(n_lanes)]
        self.streams = [torch.cuda.Stream(device=dev) for _ in range(n_lanes)]
        self.job_status = torch.zeros(nj, dtype=torch.int32, device=dev)
        self.outputs = []
        self.jobs = (Job * nj)()
        for j, st in enumerate(sets):
            J = self.jobs[j]
            J.d_xyz = st["points"].data_ptr()
            J.n = sizes[j]
            J.periodic_L = float(st.get("periodic_L", 0.0))
            J.lane = lane_of[j]
            J.nmax0 = self.job_nmax0[j]
            if st["op"] == "knn":
                k = int(st["k"])
                idx = torch.empty((sizes[j], k), dtype=torch.int32, device=dev)
                d2 = torch.empty((sizes[j], k), dtype=torch.float32, device=dev)
                J.op, J.k, J.d_idx, J.d_dist2 = JZT_OP_KNN, k, idx.data_ptr(), d2.data_ptr()
                self.outputs.append((idx, d2))
            elif st["op"] == "fof":
                lab = torch.empty(sizes[j], dtype=torch.int32, device=dev)
                J.op, J.b, J.d_labels = JZT_OP_FOF, float(st["b"]), lab.data_ptr()
                self.outputs.append(lab)
            else:
                raise ValueError(f"job {j}: op must be 'knn' or 'fof'")
        self._ws_ptrs = (ctypes.c_void_p * len(self.ws))(*[w.data_ptr() for w in self.ws])
        self._ws_bytes = (ctypes.c_size_t * len(self.ws))(*[w.numel() for w in self.ws])
        self._streams = (ctypes.c_void_p * n_lanes)(*[st.cuda_stream for st in self.streams])
        self.graph = None
        self._launch(torch.cuda.current_stream(dev))  # eager run (also warms up the kernels)
        if self.queue:
            # each job has a workspace of the default size for its N and k; the list
            # arena is an estimate (Eq. alloc_ilist), so a job that ran out of it gets
            # the size its status reports and the batch runs again
            for _ in range(3):
                grow = [j for j, c in enumerate(self.statuses()) if c == JZT_ERR_CAPACITY]
                if not grow:
                    break
                for j in grow:
                    need = status(self.ws[j])["required_bytes"]
                    self.ws[j] = torch.empty(max(int(need * 1.25), 2 * self.ws[j].numel()), dtype=torch.uint8,
                                             device=dev)
                    self._ws_ptrs[j] = self.ws[j].data_ptr()
                    self._ws_bytes[j] = self.ws[j].numel()
                self._launch(torch.cuda.current_stream(dev))
        if graph:
            torch.cuda.synchronize(dev)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, capture_error_mode="relaxed"):
                self._launch(torch.cuda.current_stream(dev))
            self.graph = g

    def _launch(self, stream):
        if self.queue:
            _check(lib.jzt_batch_run_queue(self.jobs, len(self.sets), _params(self.params), self._ws_ptrs,
                                           self._ws_bytes, self._streams, self.n_lanes,
                                           ctypes.c_void_p(stream.cuda_stream),
                                           ctypes.c_void_p(self.scratch.data_ptr()), self.scratch.numel(),
                                           ctypes.c_void_p(self.job_status.data_ptr())))
            return
        _check(lib.jzt_batch_run(self.jobs, len(self.sets), _params(self.params), self._ws_ptrs,
                                 self._ws_bytes, self._streams, self.n_lanes,
                                 ctypes.c_void_p(stream.cuda_stream),
                                 ctypes.c_void_p(self.job_status.data_ptr())))

    def run(self):
        """Enqueue the whole batch on the current stream (graph replay when captured)."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self._launch(torch.cuda.current_stream())

    def statuses(self):
        """Per-job device status codes (synchronises)."""
        return self.job_status.cpu().tolist()
