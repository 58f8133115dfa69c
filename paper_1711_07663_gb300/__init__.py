"""Python binding of libdirectcut, the GB300 (sm_103a) parallel direct cut.

Argument marshalling only: every step of the cut runs in the CUDA library
(include/directcut.h documents the operation, layouts and errors).  The
functions keep the C names (dc_create, dc_cut, dc_cut_batch, dc_submit,
dc_poll, dc_get_stats, dc_destroy); ``Context`` wraps them for convenience.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA); the
binding passes their addresses and whether they live on the device.  There is
no CPU fallback: importing works without a GPU, but any call that needs the
library raises if libdirectcut.so is missing or no CUDA device is present.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = [
    "DC_HOLE", "DC_FIELD", "DC_FRINGE", "DC_FP64", "DC_FP32_RECHECK", "DC_HEURISTIC", "DirectCutError", "load",
    "lib_path",
    "dc_create", "dc_cut", "dc_cut_batch", "dc_submit", "dc_poll", "dc_get_stats", "dc_destroy",
    "dc_last_error", "dc_version", "dc_cut_noalloc", "Context", "EXPORTED",
    "DC_WALL", "DC_OVERSET", "dc_blank_union", "dc_ab_faces", "dc_unblank", "structured_neighbours",
    "dc_get_tuning", "dc_set_tuning", "dc_autotune", "PointLocator", "dc_fail_alloc",
]

DC_OK, DC_PENDING = 0, 1
DC_EINVAL, DC_ENOMEM, DC_ECUDA, DC_EBUSY, DC_ETIMEDOUT, DC_ENOTFOUND, DC_ECANCELED, DC_EINTERNAL = range(-1, -9, -1)
DC_HOLE, DC_FIELD, DC_FRINGE = 0, 1, -1
DC_FP64, DC_FP32_RECHECK, DC_HEURISTIC = 0, 1, 2

EXPORTED = ("dc_config_default", "dc_create", "dc_cut", "dc_cut_batch", "dc_submit", "dc_poll", "dc_get_stats",
            "dc_destroy", "dc_last_error", "dc_version", "dc_cut_noalloc", "dc_blank_union", "dc_ab_faces",
            "dc_unblank", "dc_get_tuning", "dc_set_tuning", "dc_autotune", "dc_pc_create", "dc_pc_locate",
            "dc_pc_get_stats", "dc_pc_destroy", "dc_fail_alloc")
DC_WALL, DC_OVERSET = 0, 1

_HERE = os.path.dirname(os.path.abspath(__file__))


def lib_path() -> str:
    return os.path.join(_HERE, "_build", "libdirectcut.so")


class DirectCutError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"directcut status {status}: {message}")
        self.status = status


class dc_mesh_desc(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32), ("n_elem", ctypes.c_int64), ("nodes", ctypes.c_void_p),
                ("nodes_on_device", ctypes.c_int32)]


class dc_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("precision", ctypes.c_int32), ("mem_budget_bytes", ctypes.c_size_t),
                ("tol", ctypes.c_double), ("holemap_cells", ctypes.c_int32), ("bin_cubes", ctypes.c_int32),
                ("max_inflight", ctypes.c_int32), ("profile", ctypes.c_int32), ("reserve_faces", ctypes.c_int32)]


class dc_request(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int32), ("n_faces", ctypes.c_int64), ("face_nodes", ctypes.c_void_p),
                ("pose", ctypes.c_void_p), ("flags_out", ctypes.c_void_p), ("dist_out", ctypes.c_void_p),
                ("on_device", ctypes.c_int32), ("async_", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("fp32_dist_out", ctypes.c_void_p)]


class dc_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("n_elem", "n_candidates", "n_fringe", "n_hole", "n_field",
                                             "faces_visited", "pairs_bulk", "pairs_recheck", "fallbacks",
                                             "holemap_rows_undecided")] + \
               [(n, ctypes.c_float) for n in ("ms_surface", "ms_holemap", "ms_classify", "ms_exact", "ms_redo",
                                                  "ms_total")] + \
               [(n, ctypes.c_int64) for n in ("near_tasks", "n_full_search", "near_pairs_full", "heur_rescans",
                                              "heur_resolves")]


class dc_tuning(ctypes.Structure):
    _fields_ = [("cubes_per_edge", ctypes.c_float), ("bin_cubes", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("cands_per_warp", ctypes.c_int32), ("ms", ctypes.c_float)]


class dc_pc_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("n_points", "n_found", "candidates", "fp64_steps", "tree_depth")]


_lib = None
_lock = threading.Lock()


def load(build_if_missing: bool = False):
    """Load libdirectcut.so (built in-tree by paper_1711_07663_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise DirectCutError(DC_EINVAL, f"{path} is missing: run paper_1711_07663_gb300.build.build() "
                                                "(the CUDA library is required; there is no CPU fallback)")
            from . import build as _b
            _b.build()
        L = ctypes.CDLL(path)
        P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.dc_config_default.argtypes = [ctypes.POINTER(dc_config)]
        L.dc_config_default.restype = i32
        L.dc_create.argtypes = [ctypes.POINTER(dc_config), ctypes.POINTER(dc_mesh_desc), i32, ctypes.POINTER(P)]
        L.dc_create.restype = i32
        L.dc_cut.argtypes = [P, i32, ctypes.POINTER(dc_request)]
        L.dc_cut.restype = i32
        L.dc_cut_batch.argtypes = [P, i32, ctypes.POINTER(i32), ctypes.POINTER(dc_request)]
        L.dc_cut_batch.restype = i32
        L.dc_submit.argtypes = [P, i32, ctypes.POINTER(dc_request), ctypes.POINTER(ctypes.c_uint64)]
        L.dc_submit.restype = i32
        L.dc_poll.argtypes = [P, ctypes.c_uint64, i64]
        L.dc_poll.restype = i32
        L.dc_get_stats.argtypes = [P, ctypes.POINTER(dc_stats)]
        L.dc_get_stats.restype = i32
        L.dc_destroy.argtypes = [P]
        L.dc_destroy.restype = None
        L.dc_last_error.argtypes = [P]
        L.dc_last_error.restype = ctypes.c_char_p
        L.dc_version.argtypes = []
        L.dc_version.restype = ctypes.c_char_p
        L.dc_fail_alloc.argtypes = [i64]
        L.dc_fail_alloc.restype = i64
        L.dc_cut_noalloc.argtypes = [i32, i64, P, i32, i64, P, P, ctypes.c_double, P, P, P]
        L.dc_cut_noalloc.restype = i32
        L.dc_blank_union.argtypes = [i32, ctypes.POINTER(P), ctypes.POINTER(i32), i64, P, P]
        L.dc_blank_union.restype = i32
        L.dc_ab_faces.argtypes = [i64, P, P, P, ctypes.POINTER(i64), P]
        L.dc_ab_faces.restype = i32
        L.dc_unblank.argtypes = [i32, i64, P, P, P, P, P, ctypes.POINTER(i64), P]
        L.dc_unblank.restype = i32
        L.dc_get_tuning.argtypes = [P, ctypes.POINTER(dc_tuning)]
        L.dc_get_tuning.restype = i32
        L.dc_set_tuning.argtypes = [P, ctypes.POINTER(dc_tuning)]
        L.dc_set_tuning.restype = i32
        L.dc_autotune.argtypes = [P, i32, ctypes.POINTER(i32), ctypes.POINTER(dc_request), i32,
                                  ctypes.POINTER(dc_tuning), ctypes.POINTER(i32)]
        L.dc_autotune.restype = i32
        L.dc_pc_create.argtypes = [i32, i32, i64, P, i32, ctypes.POINTER(P)]
        L.dc_pc_create.restype = i32
        L.dc_pc_locate.argtypes = [P, i64, P, P, P, P, i32, P]
        L.dc_pc_locate.restype = i32
        L.dc_pc_get_stats.argtypes = [P, ctypes.POINTER(dc_pc_stats)]
        L.dc_pc_get_stats.restype = i32
        L.dc_pc_destroy.argtypes = [P]
        L.dc_pc_destroy.restype = None
        _lib = L
        return L


def dc_last_error(ctx=None) -> str:
    """The calling thread's last error message (messages are per thread; ctx
    may be given or not)."""
    return load().dc_last_error(ctx).decode()


def dc_version() -> str:
    return load().dc_version().decode()


def dc_fail_alloc(after: int) -> int:
    """Arm (after >= 0) or disarm (after < 0) a one-shot failure of the
    library's allocation `after` allocations from now; returns the number of
    device and pinned-host allocations the library has made so far."""
    return int(load().dc_fail_alloc(int(after)))


def _check(st: int) -> int:
    if st < 0:
        raise DirectCutError(st, dc_last_error())
    return st


def _addr(x, dtype):
    """(address, on_device, keepalive) of a contiguous numpy array or torch tensor."""
    if x is None:
        return None, False, None
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        import torch
        want = {np.float64: torch.float64, np.float32: torch.float32, np.int8: torch.int8, np.uint8: torch.uint8,
                np.int64: torch.int64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError(f"tensor must be contiguous {want}")
        return x.data_ptr(), bool(x.is_cuda), x
    a = np.asarray(x)
    if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"array must be C-contiguous {np.dtype(dtype)}")
    return a.ctypes.data, False, a


def make_config(**kw) -> dc_config:
    cfg = dc_config()
    _check(load().dc_config_default(ctypes.byref(cfg)))
    for k, v in kw.items():
        if v is not None:
            setattr(cfg, k, v)
    return cfg


def dc_create(meshes, **cfg_kw):
    """meshes: list of (p, nodes) with nodes [n_elem][(p+1)^3][3] float64.
    Returns an opaque context handle (int)."""
    descs = (dc_mesh_desc * len(meshes))()
    keep = []
    for i, (p, nodes) in enumerate(meshes):
        ptr, dev, k = _addr(nodes, np.float64)
        keep.append(k)
        n_elem = (k.shape[0] if hasattr(k, "shape") else len(k))
        descs[i].p, descs[i].n_elem, descs[i].nodes, descs[i].nodes_on_device = int(p), int(n_elem), ptr, int(dev)
    cfg = make_config(**cfg_kw)
    h = ctypes.c_void_p()
    _check(load().dc_create(ctypes.byref(cfg), descs, len(meshes), ctypes.byref(h)))
    return h.value


def _request(q, faces, flags_out, dist_out=None, pose=None, stream=None, async_=False, fp32_dist_out=None):
    r = dc_request()
    fp, fdev, fk = _addr(faces, np.float64)
    op, odev, ok = _addr(flags_out, np.int8)
    dp, ddev, dk = _addr(dist_out, np.float64)
    sp, sdev, sk = _addr(fp32_dist_out, np.float32)
    if dist_out is not None and ddev != odev:
        raise ValueError("flags_out and dist_out must live in the same memory")
    if fp32_dist_out is not None and sdev != odev:
        raise ValueError("flags_out and fp32_dist_out must live in the same memory")
    if fdev != odev:
        raise ValueError("face nodes and outputs must both be host or both be device memory")
    pk = None
    if pose is not None:
        pk = np.ascontiguousarray(np.asarray(pose, dtype=np.float64).reshape(12))
    r.q = int(q)
    r.n_faces = int(fk.shape[0])
    r.face_nodes = fp
    r.pose = None if pk is None else pk.ctypes.data
    r.flags_out = op
    r.dist_out = dp
    r.on_device = int(fdev)
    r.async_ = int(bool(async_))
    r.stream = None if stream is None else int(stream)
    r.fp32_dist_out = sp
    return r, (fk, ok, dk, pk, sk)


def dc_cut(ctx, mesh, q, faces, flags_out, dist_out=None, pose=None, stream=None, async_=False, fp32_dist_out=None):
    r, keep = _request(q, faces, flags_out, dist_out, pose, stream, async_, fp32_dist_out)
    _check(load().dc_cut(ctx, int(mesh), ctypes.byref(r)))


def dc_cut_batch(ctx, meshes, requests):
    """requests: list of dicts with keys q, faces, flags_out[, dist_out, pose,
    fp32_dist_out, stream] (the batch runs on the first request's stream)."""
    n = len(requests)
    arr = (dc_request * n)()
    keep = []
    for i, rq in enumerate(requests):
        r, k = _request(rq["q"], rq["faces"], rq["flags_out"], rq.get("dist_out"), rq.get("pose"),
                        stream=rq.get("stream"), fp32_dist_out=rq.get("fp32_dist_out"))
        arr[i] = r
        keep.append(k)
    ms = (ctypes.c_int32 * n)(*[int(m) for m in meshes])
    _check(load().dc_cut_batch(ctx, n, ms, arr))


def dc_submit(ctx, mesh, q, faces, flags_out, dist_out=None, pose=None):
    r, keep = _request(q, faces, flags_out, dist_out, pose)
    t = ctypes.c_uint64()
    _check(load().dc_submit(ctx, int(mesh), ctypes.byref(r), ctypes.byref(t)))
    return t.value


def dc_poll(ctx, ticket, timeout_us=0):
    """DC_OK (0) when done, DC_PENDING (1) when not; raises on errors."""
    return _check(load().dc_poll(ctx, int(ticket), int(timeout_us)))


def dc_get_stats(ctx) -> dict:
    s = dc_stats()
    _check(load().dc_get_stats(ctx, ctypes.byref(s)))
    return {n: getattr(s, n) for n, _ in dc_stats._fields_}


def dc_cut_noalloc(p, nodes, q, faces, flags_out, dist_out=None, pose=None, tol=0.0, stream=None):
    """Allocation-free cut (device tensors only): see dc_cut_noalloc in the
    header.  For callers that may not allocate device memory when they cut
    (allocation-free real-time loops, hosts whose own allocator owns the
    GPU's memory).  Shapes are checked here, so that a short output or a
    flattened node array is a ValueError instead of an out-of-bounds access
    on the device."""
    np_, ndev, nk = _addr(nodes, np.float64)
    fp, fdev, fk = _addr(faces, np.float64)
    op, odev, ok = _addr(flags_out, np.int8)
    dp, ddev, dk = _addr(dist_out, np.float64)
    if not (ndev and fdev and odev and (dist_out is None or ddev)):
        raise ValueError("dc_cut_noalloc takes device tensors only")
    p, q = int(p), int(q)
    if tuple(nk.shape[1:]) != ((p + 1) ** 3, 3) or nk.dim() != 3:
        raise ValueError(f"nodes must have shape [n_elem][{(p + 1) ** 3}][3] for p={p}, got {tuple(nk.shape)}")
    if tuple(fk.shape[1:]) != ((q + 1) ** 2, 3) or fk.dim() != 3:
        raise ValueError(f"faces must have shape [n_faces][{(q + 1) ** 2}][3] for q={q}, got {tuple(fk.shape)}")
    n_elem = int(nk.shape[0])
    if ok.numel() < n_elem:
        raise ValueError(f"flags_out holds {ok.numel()} entries, {n_elem} needed")
    if dk is not None and dk.numel() < n_elem:
        raise ValueError(f"dist_out holds {dk.numel()} entries, {n_elem} needed")
    pk = None if pose is None else np.ascontiguousarray(np.asarray(pose, dtype=np.float64).reshape(12))
    _check(load().dc_cut_noalloc(p, n_elem, np_, q, int(fk.shape[0]), fp,
                                 None if pk is None else pk.ctypes.data, float(tol), op, dp,
                                 None if stream is None else int(stream)))


def _dev(x, dtype, what):
    p, dev, k = _addr(x, dtype)
    if not dev:
        raise ValueError(f"{what} must be a device tensor")
    return p, k


def dc_blank_union(flags, kinds, iblank_out, stream=None):
    """iblank (1 kept, 0 removed) of several cuts: see dc_blank_union in the header."""
    ptrs = [_dev(f, np.int8, "flags")[0] for f in flags]
    ob, ok = _dev(iblank_out, np.int8, "iblank_out")
    arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
    kk = (ctypes.c_int32 * len(kinds))(*[int(k) for k in kinds])
    _check(load().dc_blank_union(len(ptrs), arr, kk, int(ok.shape[0]), ob, None if stream is None else int(stream)))


def dc_ab_faces(iblank, neighbours, ab_mask, stream=None) -> int:
    """Artificial-boundary face masks; returns the number of such faces."""
    ib, ik = _dev(iblank, np.int8, "iblank")
    nb, _ = _dev(neighbours, np.int64, "neighbours")
    mb, _ = _dev(ab_mask, np.uint8, "ab_mask")
    n = ctypes.c_int64(0)
    _check(load().dc_ab_faces(int(ik.shape[0]), ib, nb, mb, ctypes.byref(n), None if stream is None else int(stream)))
    return n.value


def dc_unblank(kind, iblank_prev, flags_t, flags_tp, iblank_out, unblank_out, stream=None) -> int:
    """The unblank step for one cut kind; returns the number of elements to unblank."""
    pp, pk = _dev(iblank_prev, np.int8, "iblank_prev")
    tp_, _ = _dev(flags_t, np.int8, "flags_t")
    tq, _ = _dev(flags_tp, np.int8, "flags_tp")
    ob, _ = _dev(iblank_out, np.int8, "iblank_out")
    ub, _ = _dev(unblank_out, np.uint8, "unblank_out")
    n = ctypes.c_int64(0)
    _check(load().dc_unblank(int(kind), int(pk.shape[0]), pp, tp_, tq, ob, ub, ctypes.byref(n),
                             None if stream is None else int(stream)))
    return n.value


def structured_neighbours(nx, ny, nz) -> np.ndarray:
    """Face neighbours [n][6] int64 of the hexes of an nx*ny*nz block numbered
    ex + nx*(ey + ny*ez), faces xi-, xi+, eta-, eta+, zeta-, zeta+; -1 on the
    block boundary (the input dc_ab_faces takes for a structured grid)."""
    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    e = (ex + nx * (ey + ny * ez)).reshape(-1).astype(np.int64)
    ex, ey, ez = ex.reshape(-1), ey.reshape(-1), ez.reshape(-1)
    out = np.full((e.size, 6), -1, dtype=np.int64)
    out[:, 0] = np.where(ex > 0, e - 1, -1)
    out[:, 1] = np.where(ex < nx - 1, e + 1, -1)
    out[:, 2] = np.where(ey > 0, e - nx, -1)
    out[:, 3] = np.where(ey < ny - 1, e + nx, -1)
    out[:, 4] = np.where(ez > 0, e - nx * ny, -1)
    out[:, 5] = np.where(ez < nz - 1, e + nx * ny, -1)
    return out


def dc_destroy(ctx) -> None:
    if ctx:
        load().dc_destroy(ctx)


def _tuning_dict(t):
    return {n: getattr(t, n) for n, _ in dc_tuning._fields_}


def dc_get_tuning(ctx) -> dict:
    t = dc_tuning()
    _check(load().dc_get_tuning(ctx, ctypes.byref(t)))
    return _tuning_dict(t)


def dc_set_tuning(ctx, **kw):
    """Change some launch shapes (keys of dc_tuning); the others stay."""
    t = dc_tuning()
    _check(load().dc_get_tuning(ctx, ctypes.byref(t)))
    for k, v in kw.items():
        if k not in dict(dc_tuning._fields_):
            raise KeyError(k)
        setattr(t, k, v)
    _check(load().dc_set_tuning(ctx, ctypes.byref(t)))


def dc_autotune(ctx, meshes, requests, repeats=3):
    """Sweep the launch shapes on a batch (requests as for dc_cut_batch), keep
    the fastest on the context; returns (setting dict with its median ms,
    number of settings timed)."""
    n = len(requests)
    arr = (dc_request * n)()
    keep = []
    for i, rq in enumerate(requests):
        r, k = _request(rq["q"], rq["faces"], rq["flags_out"], rq.get("dist_out"), rq.get("pose"),
                        stream=rq.get("stream"))
        arr[i] = r
        keep.append(k)
    ms = (ctypes.c_int32 * n)(*[int(m) for m in meshes])
    best = dc_tuning()
    trials = ctypes.c_int32(0)
    _check(load().dc_autotune(ctx, n, ms, arr, int(repeats), ctypes.byref(best), ctypes.byref(trials)))
    return _tuning_dict(best), trials.value


class PointLocator:
    """Donor search on one grid: PointLocator(p, nodes[, device]); locate(pts,
    pose=None) -> (donor int64 [n], ref float64 [n][3]) for host arrays, or
    writes into given device tensors."""

    def __init__(self, p, nodes, device=0):
        np_, ndev, keep = _addr(nodes, np.float64)
        h = ctypes.c_void_p()
        _check(load().dc_pc_create(int(device), int(p), int(keep.shape[0]), np_, int(ndev), ctypes.byref(h)))
        self.handle = h
        self.n_elem = int(keep.shape[0])

    def locate(self, pts, pose=None, donor_out=None, ref_out=None, stream=None):
        pp, pdev, pk = _addr(pts, np.float64)
        n = int(pk.shape[0]) if pk.ndim > 1 else int(pk.shape[0]) // 3
        if donor_out is None:
            if pdev:
                import torch
                donor_out = torch.empty(n, dtype=torch.int64, device=pts.device)
                ref_out = torch.empty((n, 3), dtype=torch.float64, device=pts.device)
            else:
                donor_out = np.empty(n, dtype=np.int64)
                ref_out = np.empty((n, 3), dtype=np.float64)
        dp, ddev, dk = _addr(donor_out, np.int64)
        rp, rdev, rk = _addr(ref_out, np.float64)
        if not (pdev == ddev == rdev):
            raise ValueError("points, donor_out and ref_out must all be host arrays or all device tensors")
        pk_ = None if pose is None else np.ascontiguousarray(np.asarray(pose, dtype=np.float64).reshape(12))
        _check(load().dc_pc_locate(self.handle, n, pp, None if pk_ is None else pk_.ctypes.data, dp, rp, int(pdev),
                                   None if stream is None else int(stream)))
        return donor_out, ref_out

    def stats(self):
        s = dc_pc_stats()
        _check(load().dc_pc_get_stats(self.handle, ctypes.byref(s)))
        return {n: getattr(s, n) for n, _ in dc_pc_stats._fields_}

    def close(self):
        if self.handle:
            load().dc_pc_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """Owning wrapper: Context([(p, nodes), ...], precision=..., ...)."""

    def __init__(self, meshes, **cfg):
        self.meshes = [(int(p), nodes) for p, nodes in meshes]
        self.n_elem = [int(n.shape[0]) for _, n in self.meshes]
        self.handle = dc_create(self.meshes, **cfg)

    def cut(self, mesh, q, faces, flags_out=None, dist_out=None, pose=None, stream=None, async_=False,
            fp32_dist_out=None):
        if flags_out is None:
            n = self.n_elem[mesh] if 0 <= mesh < len(self.n_elem) else 1
            flags_out = np.empty(n, dtype=np.int8)
        dc_cut(self.handle, mesh, q, faces, flags_out, dist_out, pose, stream, async_, fp32_dist_out)
        return flags_out

    def cut_batch(self, meshes, requests):
        dc_cut_batch(self.handle, meshes, requests)

    def submit(self, mesh, q, faces, flags_out, dist_out=None, pose=None):
        return dc_submit(self.handle, mesh, q, faces, flags_out, dist_out, pose)

    def poll(self, ticket, timeout_us=0):
        return dc_poll(self.handle, ticket, timeout_us)

    def stats(self):
        return dc_get_stats(self.handle)

    def tuning(self):
        return dc_get_tuning(self.handle)

    def set_tuning(self, **kw):
        dc_set_tuning(self.handle, **kw)

    def autotune(self, meshes, requests, repeats=3):
        return dc_autotune(self.handle, meshes, requests, repeats)

    def close(self):
        if self.handle:
            dc_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
