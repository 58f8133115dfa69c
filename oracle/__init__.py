"""Python access to the FP64 CPU oracle (oracle/oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and by
the benchmark's CPU-baseline leg.  The CUDA library never imports it and shares
no code with it.  See oracle.c for what is computed and which passage of the
paper each step follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None

HOLE, FIELD, FRINGE = 0, 1, -1


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, OpenMP, no FMA
    contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            d, i32, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
            P = ctypes.c_void_p
            L.orc_tritri.restype = d
            L.orc_tritri.argtypes = [P, P, P, P]
            L.orc_pt_tri.restype = d
            L.orc_pt_tri.argtypes = [P, P, P]
            L.orc_seg_seg.restype = d
            L.orc_seg_seg.argtypes = [P, P, P, P, P, P]
            L.orc_elem_tris.restype = None
            L.orc_elem_tris.argtypes = [i32, P, P]
            L.orc_face_tris.restype = None
            L.orc_face_tris.argtypes = [i32, P, P]
            L.orc_winding.restype = d
            L.orc_winding.argtypes = [P, i64, P]
            L.orc_signed_volume.restype = d
            L.orc_signed_volume.argtypes = [i64, P]
            L.orc_apply_pose.restype = None
            L.orc_apply_pose.argtypes = [i64, P, P, P]
            L.orc_box_dist.restype = d
            L.orc_box_dist.argtypes = [P, P]
            L.orc_point_surface.restype = d
            L.orc_point_surface.argtypes = [P, i64, P, P]
            L.orc_cut.restype = i32
            L.orc_cut.argtypes = [i32, i64, P, i32, i64, P, P, d, i32, P, i64, P, P, P, P, i32]
            L.orc_obb.restype = None
            L.orc_obb.argtypes = [P, i32, P, P, P]
            L.orc_approx_dist.restype = d
            L.orc_approx_dist.argtypes = [P, P, P, P]
            L.orc_pass1.restype = d
            L.orc_pass1.argtypes = [i32, P, i32, P, d, ctypes.POINTER(i32), ctypes.POINTER(d)]
            L.orc_lagrange.restype = None
            L.orc_lagrange.argtypes = [i32, d, P, P]
            L.orc_map.restype = None
            L.orc_map.argtypes = [i32, P, P, P, P]
            L.orc_newton.restype = i32
            L.orc_newton.argtypes = [i32, P, P, d, P, ctypes.POINTER(d), ctypes.POINTER(i32)]
            L.orc_locate.restype = i32
            L.orc_locate.argtypes = [i32, i64, P, i64, P, P, P, P, P, i32]
            L.orc_pair_dist.restype = i32
            L.orc_pair_dist.argtypes = [i32, i64, P, i32, i64, P, i64, P, P, P, i32]
            L.orc_heuristic.restype = i32
            L.orc_heuristic.argtypes = [i32, i64, P, i32, i64, P, P, d, i32, i32, P, i64, P, P, P, P, i32]
            _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


def tritri(A, B):
    """Distance between closed triangles A, B (3x3 each) and the closest points."""
    A, B = _f64(A), _f64(B)
    ca, cb = np.zeros(3), np.zeros(3)
    d = lib().orc_tritri(_ptr(A), _ptr(B), _ptr(ca), _ptr(cb))
    return d, ca, cb


def pt_tri(P, T):
    P, T = _f64(P), _f64(T)
    c = np.zeros(3)
    return lib().orc_pt_tri(_ptr(P), _ptr(T), _ptr(c)), c


def seg_seg(p0, p1, q0, q1):
    a = [_f64(x) for x in (p0, p1, q0, q1)]
    cp, cq = np.zeros(3), np.zeros(3)
    d = lib().orc_seg_seg(*[_ptr(x) for x in a], _ptr(cp), _ptr(cq))
    return d, cp, cq


def elem_tris(p, nodes):
    nodes = _f64(nodes)
    out = np.zeros((12 * p * p, 3, 3))
    lib().orc_elem_tris(p, _ptr(nodes), _ptr(out))
    return out


def face_tris(q, fnodes):
    fnodes = _f64(fnodes)
    out = np.zeros((2 * q * q, 3, 3))
    lib().orc_face_tris(q, _ptr(fnodes), _ptr(out))
    return out


def surface_tris(q, faces):
    faces = _f64(faces)
    return np.concatenate([face_tris(q, f) for f in faces], axis=0)


def winding(P, tris):
    P, tris = _f64(P), _f64(tris)
    return lib().orc_winding(_ptr(P), tris.shape[0], _ptr(tris))


def signed_volume(tris):
    tris = _f64(tris)
    return lib().orc_signed_volume(tris.shape[0], _ptr(tris))


def apply_pose(faces, pose):
    faces = _f64(faces)
    if pose is None:
        return faces.copy()
    pose = _f64(np.asarray(pose).reshape(3, 4))
    out = np.empty_like(faces)
    lib().orc_apply_pose(faces.size // 3, _ptr(faces), _ptr(pose), _ptr(out))
    return out


def box_dist(b1, b2):
    b1, b2 = _f64(b1), _f64(b2)
    return lib().orc_box_dist(_ptr(b1), _ptr(b2))


def point_surface(P, tris):
    P, tris = _f64(P), _f64(tris)
    w = ctypes.c_double(0.0)
    d = lib().orc_point_surface(_ptr(P), tris.shape[0], _ptr(tris), ctypes.byref(w))
    return d, w.value


STAT_NAMES = ("tritri_tests", "s_star_pairs", "s_star_tri_pairs", "undecidable", "paper_rule_disagree",
              "fringe", "hole", "field")


def cut(p, nodes, q, faces, pose=None, tol=1e-7, brute=False, ids=None, nthreads=0):
    """Classify elements: returns (flags int8, dist f64, paper_flags int8, stats dict).
    ``ids`` selects a subset of elements (outputs follow its order)."""
    nodes, faces = _f64(nodes), _f64(faces)
    n_elem = nodes.shape[0]
    ids_arr = None if ids is None else np.ascontiguousarray(ids, dtype=np.int64)
    nev = n_elem if ids_arr is None else ids_arr.shape[0]
    flags = np.zeros(nev, dtype=np.int8)
    pflags = np.zeros(nev, dtype=np.int8)
    dist = np.zeros(nev, dtype=np.float64)
    stats = np.zeros(8, dtype=np.int64)
    pose_arr = None if pose is None else _f64(np.asarray(pose).reshape(3, 4))
    rc = lib().orc_cut(p, n_elem, _ptr(nodes), q, faces.shape[0], _ptr(faces), _ptr(pose_arr), float(tol),
                       1 if brute else 0, _ptr(ids_arr), nev, _ptr(flags), _ptr(dist), _ptr(pflags), _ptr(stats),
                       int(nthreads))
    if rc != 0:
        raise ValueError("orc_cut rejected its arguments")
    return flags, dist, pflags, dict(zip(STAT_NAMES, (int(x) for x in stats)))


def pair_dist(p, nodes, q, posed_faces, elem, face, nthreads=0):
    """d(E, F) of element-face pairs: the minimum closed-triangle distance
    between element elem[k]'s boundary triangles and face face[k]'s triangles
    (faces already posed)."""
    nodes, posed_faces = _f64(nodes), _f64(posed_faces)
    elem = np.ascontiguousarray(elem, dtype=np.int64)
    face = np.ascontiguousarray(face, dtype=np.int64)
    out = np.zeros(elem.shape[0], dtype=np.float64)
    rc = lib().orc_pair_dist(p, nodes.shape[0], _ptr(nodes), q, posed_faces.shape[0], _ptr(posed_faces),
                             elem.shape[0], _ptr(elem), _ptr(face), _ptr(out), int(nthreads))
    if rc != 0:
        raise ValueError("orc_pair_dist rejected its arguments")
    return out


# ----------------------------------------------------------------- the paper's truncating variant
MARGIN_NAMES = ("key_gap", "corner_gap", "d1_gap", "zero_tie_key_gap", "d2_tol_gap", "side_cos")


def obb(pts):
    """OBB of points [n][3]: (R rows = axes, box [6] in those axes, centroid)."""
    pts = _f64(pts)
    R = np.zeros(9)
    box = np.zeros(6)
    cg = np.zeros(3)
    lib().orc_obb(_ptr(pts), pts.shape[0], _ptr(R), _ptr(box), _ptr(cg))
    return R.reshape(3, 3), box, cg


def approx_dist(R, Be, ecg, Xf):
    """Alg. cp0 key of a face (corner nodes Xf [4][3]) against an element OBB."""
    R, Be, ecg, Xf = _f64(R), _f64(Be), _f64(ecg), _f64(Xf)
    return lib().orc_approx_dist(_ptr(R), _ptr(Be), _ptr(ecg), _ptr(Xf))


def pass1(p, enodes, q, fnodes, tol=1e-7):
    """Alg. cp1 on one element-face pair: (D1, corner, corner gap)."""
    enodes, fnodes = _f64(enodes), _f64(fnodes)
    c = ctypes.c_int(0)
    g = ctypes.c_double(0.0)
    d1 = lib().orc_pass1(p, _ptr(enodes), q, _ptr(fnodes), float(tol), ctypes.byref(c), ctypes.byref(g))
    return d1, c.value, g.value


def heuristic(p, nodes, q, faces, pose=None, tol=1e-7, nf1=16, nf2=4, ids=None, nthreads=0):
    """The paper's truncating variant: (flags int8, flagset uint8, dist f64,
    margins [n][6]); flagset bit (flag + 1) marks every flag an exact tie at the
    second truncation allows."""
    nodes, faces = _f64(nodes), _f64(faces)
    ids_arr = None if ids is None else np.ascontiguousarray(ids, dtype=np.int64)
    nev = nodes.shape[0] if ids_arr is None else ids_arr.shape[0]
    flags = np.zeros(nev, dtype=np.int8)
    fset = np.zeros(nev, dtype=np.uint8)
    dist = np.zeros(nev, dtype=np.float64)
    margins = np.zeros((nev, 6), dtype=np.float64)
    pose_arr = None if pose is None else _f64(np.asarray(pose).reshape(3, 4))
    rc = lib().orc_heuristic(p, nodes.shape[0], _ptr(nodes), q, faces.shape[0], _ptr(faces), _ptr(pose_arr),
                             float(tol), int(nf1), int(nf2), _ptr(ids_arr), nev, _ptr(flags), _ptr(fset), _ptr(dist),
                             _ptr(margins), int(nthreads))
    if rc != 0:
        raise ValueError("orc_heuristic rejected its arguments")
    return flags, fset, dist, margins


# ----------------------------------------------------------------- donor search (point connectivity)
def lagrange(p, x):
    """Lagrange basis on the p+1 equispaced nodes of [-1,1] at x: (l, dl/dx)."""
    l, dl = np.zeros(p + 1), np.zeros(p + 1)
    lib().orc_lagrange(p, float(x), _ptr(l), _ptr(dl))
    return l, dl


def iso_map(p, enodes, xi):
    """x(xi) and the Jacobian dx/dxi (3x3, row = component) of one element."""
    enodes, xi = _f64(enodes), _f64(xi)
    x, J = np.zeros(3), np.zeros(9)
    lib().orc_map(p, _ptr(enodes), _ptr(xi), _ptr(x), _ptr(J))
    return x, J.reshape(3, 3)


def newton(p, enodes, x, h):
    """The clamped Newton inversion from xi = 0: (converged, xi, residual, iterations)."""
    enodes, x = _f64(enodes), _f64(x)
    xi = np.zeros(3)
    r = ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    ok = lib().orc_newton(p, _ptr(enodes), _ptr(x), float(h), _ptr(xi), ctypes.byref(r), ctypes.byref(it))
    return bool(ok), xi, r.value, it.value


def locate(p, nodes, pts, pose=None, nthreads=0):
    """Donor element (-1: none) and reference coordinates of each point, and
    the acceptance margins [n][2] (residual gap, reference gap)."""
    nodes, pts = _f64(nodes), _f64(pts).reshape(-1, 3)
    n = pts.shape[0]
    donor = np.zeros(n, dtype=np.int64)
    ref = np.zeros((n, 3))
    margins = np.zeros((n, 2))
    pose_arr = None if pose is None else _f64(np.asarray(pose).reshape(3, 4))
    rc = lib().orc_locate(p, nodes.shape[0], _ptr(nodes), n, _ptr(pts), _ptr(pose_arr), _ptr(donor), _ptr(ref),
                          _ptr(margins), int(nthreads))
    if rc != 0:
        raise ValueError("orc_locate rejected its arguments")
    return donor, ref, margins
