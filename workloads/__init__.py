"""Seeded synthetic inputs for the parallel direct cut.

This module only *builds geometry*: background hexahedral grids of order p and
closed cut surfaces made of order-q quadrilateral faces.  It holds none of the
cut's arithmetic (no distances, no bounding volumes, no classification), so the
CUDA path and the CPU oracle can both be fed from it without sharing any method
code.

Determinism across machines: every value is produced from IEEE-754 correctly
rounded operations (+, -, *, /, sqrt) and from numpy's PCG64 bit stream, both of
which are identical on x86_64 and aarch64.  The transcendental functions the
generators need (sin, cos, exp) are evaluated by the small argument-reduction +
Taylor routines below instead of the platform's libm/SIMD kernels, whose last
bits differ between machines.

Conventions (shared by the C-ABI and the oracle):
  * element nodes: float64 [n_elem][(p+1)^3][3], node (i,j,k) at
    i + (p+1)*(j + (p+1)*k), i along xi fastest (tensor-product Lagrange
    nodes, Eq. (reftophys) of the paper).
  * face nodes: float64 [n_faces][(q+1)^2][3], node (i,j) at i + (q+1)*j,
    oriented so that dx/dxi x dx/deta points out of the region to blank.
"""
from __future__ import annotations

import dataclasses
from decimal import Decimal, getcontext

import numpy as np

# --------------------------------------------------------------------------
# deterministic elementary functions (numpy, basic IEEE ops only)
# --------------------------------------------------------------------------
_PI_DIGITS = "3.14159265358979323846264338327950288419716939937510582097494459230781640628"


def _split_constant(value: Decimal, bits: int, parts: int):
    """Split ``value`` into ``parts`` doubles, the leading ones holding at most
    ``bits`` significant bits so that k*part is exact for moderate integers k."""
    out = []
    rem = value
    for i in range(parts):
        f = float(rem)
        if i < parts - 1:
            m, e = np.frexp(f)
            scale = 2.0 ** bits
            f = float(np.ldexp(np.floor(m * scale) / scale, e))
        out.append(f)
        rem = rem - Decimal(f)
    return out


getcontext().prec = 60
_PIO2 = Decimal(_PI_DIGITS) / 2
_PIO2_PARTS = _split_constant(_PIO2, 30, 3)
_LN2 = Decimal(2).ln()
_LN2_PARTS = _split_constant(_LN2, 30, 2)
PI = float(Decimal(_PI_DIGITS))


def _poly(r2, coeffs):
    acc = np.zeros_like(r2) + coeffs[-1]
    for c in coeffs[-2::-1]:
        acc = acc * r2 + c
    return acc


_SIN_C = [(-1.0) ** n / float(np.prod(np.arange(1, 2 * n + 2, dtype=np.float64))) for n in range(10)]
_COS_C = [(-1.0) ** n / float(np.prod(np.arange(1, 2 * n + 1, dtype=np.float64))) if n else 1.0 for n in range(10)]


def det_sincos(x):
    """sin(x), cos(x) for |x| < 1e5 to ~1 ulp, bit-identical on every IEEE machine."""
    x = np.asarray(x, dtype=np.float64)
    k = np.rint(x / float(_PIO2))
    r = ((x - k * _PIO2_PARTS[0]) - k * _PIO2_PARTS[1]) - k * _PIO2_PARTS[2]
    r2 = r * r
    s = r * _poly(r2, _SIN_C)
    c = _poly(r2, _COS_C)
    q = np.mod(k, 4.0)
    sin = np.where(q == 0, s, np.where(q == 1, c, np.where(q == 2, -s, -c)))
    cos = np.where(q == 0, c, np.where(q == 1, -s, np.where(q == 2, -c, s)))
    return sin, cos


def det_sin(x):
    return det_sincos(x)[0]


def det_cos(x):
    return det_sincos(x)[1]


_EXP_C = [1.0 / float(np.prod(np.arange(1, n + 1, dtype=np.float64))) if n else 1.0 for n in range(16)]


def det_exp(x):
    """exp(x) for x <= 700, bit-identical on every IEEE machine (0 below -700)."""
    x = np.asarray(x, dtype=np.float64)
    xc = np.clip(x, -700.0, 700.0)
    k = np.rint(xc / float(_LN2))
    r = (xc - k * _LN2_PARTS[0]) - k * _LN2_PARTS[1]
    e = _poly(r, _EXP_C)
    out = np.ldexp(e, k.astype(np.int64))
    return np.where(x < -700.0, 0.0, out)


# --------------------------------------------------------------------------
# random helpers
# --------------------------------------------------------------------------
def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def random_rotation(g: np.random.Generator) -> np.ndarray:
    """Uniform random rotation matrix (Shoemake's unit-quaternion construction)."""
    u1, u2, u3 = g.random(3)
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    s2, c2 = det_sincos(2.0 * PI * u2)
    s3, c3 = det_sincos(2.0 * PI * u3)
    x, y, z, w = a * s2, a * c2, b * s3, b * c3
    return np.array(
        [
            [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
            [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
            [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
        ],
        dtype=np.float64,
    )


def rotate_points(X: np.ndarray, R: np.ndarray) -> np.ndarray:
    """R @ x for every point of X [..., 3], written out elementwise (no BLAS, so
    the rounding is the same on every machine)."""
    R = np.asarray(R, dtype=np.float64)
    out = np.empty_like(X)
    for a in range(3):
        out[..., a] = (R[a, 0] * X[..., 0] + R[a, 1] * X[..., 1]) + R[a, 2] * X[..., 2]
    return out


def axis_rotation(axis, angle_rad: float) -> np.ndarray:
    """Rotation by ``angle_rad`` about unit ``axis`` (Rodrigues form)."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.sqrt(np.dot(a, a))
    s, c = det_sincos(np.float64(angle_rad))
    s, c = float(s), float(c)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]], dtype=np.float64)
    KK = np.array([[sum(K[i, k] * K[k, j] for k in range(3)) for j in range(3)] for i in range(3)])
    return np.eye(3) + s * K + (1.0 - c) * KK


# --------------------------------------------------------------------------
# background grids
# --------------------------------------------------------------------------
def hex_lattice(n: int, p: int, lo: float = -2.0, hi: float = 2.0) -> np.ndarray:
    """Equispaced global node lattice [(n*p+1)^3][3] (x fastest) of an n^3 grid of
    order-p hexes on the cube [lo, hi]^3."""
    m = n * p + 1
    t = lo + (hi - lo) * (np.arange(m, dtype=np.float64) / (n * p))
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    return np.stack([x, y, z], axis=-1).reshape(m, m, m, 3)


def gather_index(n: int, p: int) -> np.ndarray:
    """Flat lattice index [n^3][(p+1)^3] (int64) of every element node: the
    nodes of element ex + n*(ey + n*ez) are lattice.reshape(-1, 3)[index[e]]."""
    e = np.arange(n, dtype=np.int64)
    l = np.arange(p + 1, dtype=np.int64)
    ez, ey, ex = np.meshgrid(e, e, e, indexing="ij")
    lk, lj, li = np.meshgrid(l, l, l, indexing="ij")
    m = n * p + 1
    X = (ex.reshape(-1, 1) * p + li.reshape(1, -1))
    Y = (ey.reshape(-1, 1) * p + lj.reshape(1, -1))
    Z = (ez.reshape(-1, 1) * p + lk.reshape(1, -1))
    return np.ascontiguousarray((Z * m + Y) * m + X)


def gather_elements(lattice: np.ndarray, n: int, p: int) -> np.ndarray:
    """Per-element node arrays [n^3][(p+1)^3][3] gathered from the lattice, so
    nodes shared between elements are bit-identical.  Element (ex,ey,ez) is
    number ex + n*(ey + n*ez)."""
    return np.ascontiguousarray(lattice.reshape(-1, lattice.shape[-1])[gather_index(n, p)])


def jitter_lattice(lattice: np.ndarray, amp: float, g: np.random.Generator) -> np.ndarray:
    return lattice + g.uniform(-amp, amp, size=lattice.shape)


def sinusoid_lattice(lattice: np.ndarray, amp: float) -> np.ndarray:
    """x + amp*(sin(pi y) sin(pi z), sin(pi z) sin(pi x), sin(pi x) sin(pi y))."""
    sx = det_sin(PI * lattice[..., 0])
    sy = det_sin(PI * lattice[..., 1])
    sz = det_sin(PI * lattice[..., 2])
    d = np.stack([sy * sz, sz * sx, sx * sy], axis=-1)
    return lattice + amp * d


def background(n: int, p: int, *, jitter: float = 0.0, sinusoid: float = 0.0, seed: int = 0,
               lo: float = -2.0, hi: float = 2.0) -> np.ndarray:
    """An n^3 order-p background grid on [lo,hi]^3; ``jitter`` and ``sinusoid`` are
    amplitudes in units of the element size h."""
    h = (hi - lo) / n
    lat = hex_lattice(n, p, lo, hi)
    if jitter:
        lat = jitter_lattice(lat, jitter * h, rng(seed))
    if sinusoid:
        lat = sinusoid_lattice(lat, sinusoid * h)
    return gather_elements(lat, n, p)


# --------------------------------------------------------------------------
# closed cut surfaces: cubed spheres
# --------------------------------------------------------------------------
# For each cube face: (fixed axis, sign, axis of xi, axis of eta) chosen so that
# e_xi x e_eta is the outward normal of that cube face.
_CUBE_FACES = [
    (0, +1, 1, 2), (0, -1, 2, 1),
    (1, +1, 2, 0), (1, -1, 0, 2),
    (2, +1, 0, 1), (2, -1, 1, 0),
]


def cube_face_points(n: int, q: int) -> np.ndarray:
    """Integer points on the cube [-nq, nq]^3 for the 6*n*n order-q cells of a
    cubed sphere: int64 [6*n*n][(q+1)^2][3].  Shared edge/corner points carry
    identical integers, which keeps the mapped surface watertight."""
    M = n * q
    cells = []
    for ax, sg, axi, aeta in _CUBE_FACES:
        for cj in range(n):
            for ci in range(n):
                pts = np.zeros(((q + 1) ** 2, 3), dtype=np.int64)
                for j in range(q + 1):
                    for i in range(q + 1):
                        u = 2 * (ci * q + i) - M
                        v = 2 * (cj * q + j) - M
                        pt = [0, 0, 0]
                        pt[ax] = sg * M
                        pt[axi] = u
                        pt[aeta] = v
                        pts[i + (q + 1) * j] = pt
                cells.append(pts)
    return np.stack(cells)


def fibonacci_sphere(k: int, rot: np.ndarray | None = None) -> np.ndarray:
    i = np.arange(k, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / k
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * (PI * (3.0 - np.sqrt(5.0)))
    s, c = det_sincos(phi)
    pts = np.stack([r * c, r * s, z], axis=-1)
    if rot is not None:
        pts = rotate_points(pts, rot)
    return pts


def dimple_radius(xhat: np.ndarray, centres: np.ndarray, depth: float = 0.01, width: float = 0.08) -> np.ndarray:
    """1 - depth * sum_k exp(-|xhat - c_k|^2 / (2 width^2))."""
    acc = np.zeros(xhat.shape[:-1], dtype=np.float64)
    inv = 1.0 / (2.0 * width * width)
    for c in centres:
        d = xhat - c
        acc = acc + det_exp(-(d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1] + d[..., 2] * d[..., 2]) * inv)
    return 1.0 - depth * acc


def cubed_sphere(n: int, q: int, *, radius: float = 1.0, centre=(0.0, 0.0, 0.0), rot: np.ndarray | None = None,
                 dimples: np.ndarray | None = None) -> np.ndarray:
    """A closed, watertight, outward-oriented surface of 6*n*n order-q faces:
    float64 [6n^2][(q+1)^2][3].  With ``dimples`` the radius is
    radius * dimple_radius(xhat, dimples)."""
    P = cube_face_points(n, q).astype(np.float64)
    nrm = np.sqrt(P[..., 0] * P[..., 0] + P[..., 1] * P[..., 1] + P[..., 2] * P[..., 2])
    xhat = P / nrm[..., None]
    r = np.full(xhat.shape[:-1], radius, dtype=np.float64)
    if dimples is not None:
        r = radius * dimple_radius(xhat, dimples)
    X = xhat * r[..., None]
    if rot is not None:
        X = rotate_points(X, rot)
    X = X + np.asarray(centre, dtype=np.float64)
    return np.ascontiguousarray(X)


def sphere_shell(n: int, layers: int, p: int, r0: float = 1.0, r1: float = 1.6, centre=(0.0, 0.0, 0.0)) -> np.ndarray:
    """A body-fitted near-body grid around a sphere: 6*n*n*layers order-p hexes
    filling r0 <= r <= r1 (cubed-sphere cells x radial layers), float64
    [E][(p+1)^3][3] in tensor order (i, j along the cube-face cell, k radial).
    Node radii are equispaced; directions are the cubed-sphere lattice points,
    so neighbouring elements share identical nodes."""
    P = cube_face_points(n, p).astype(np.float64)
    nrm = np.sqrt(P[..., 0] * P[..., 0] + P[..., 1] * P[..., 1] + P[..., 2] * P[..., 2])
    xhat = P / nrm[..., None]                                  # [6n^2][(p+1)^2][3]
    kk = np.arange(layers * p + 1, dtype=np.float64)
    radii = r0 + (r1 - r0) * kk / (layers * p)
    out = np.empty((xhat.shape[0], layers, p + 1, (p + 1) ** 2, 3), dtype=np.float64)
    for L in range(layers):
        for k in range(p + 1):
            out[:, L, k] = xhat * radii[L * p + k]
    out = out.reshape(xhat.shape[0] * layers, (p + 1) ** 3, 3)
    return np.ascontiguousarray(out + np.asarray(centre, dtype=np.float64))


def morton_order(pts: np.ndarray, bits: int = 10) -> np.ndarray:
    """Indices that sort points along a Z-order (Morton) curve of their
    bounding box, 2^bits cells per axis."""
    lo, hi = pts.min(axis=0), pts.max(axis=0)
    cell = np.minimum(((pts - lo) / np.maximum(hi - lo, 1e-300) * (1 << bits)).astype(np.int64), (1 << bits) - 1)
    code = np.zeros(pts.shape[0], dtype=np.int64)
    for b in range(bits):
        for a in range(3):
            code |= ((cell[:, a] >> b) & 1) << (3 * b + a)
    return np.argsort(code, kind="stable")


def shell_points(count: int, r0: float, r1: float, seed: int, centre=(0.0, 0.0, 0.0), order: str = "random") -> np.ndarray:
    """Seeded points spread over the shell r0 <= r <= r1 (uniform direction,
    uniform radius): float64 [count][3].  order="morton" lists them along a
    space-filling curve, as receptor points come face by face from a grid."""
    g = rng(seed)
    d = g.normal(size=(count, 3))
    d /= np.sqrt((d * d).sum(axis=1))[:, None]
    r = g.uniform(r0, r1, size=count)
    pts = d * r[:, None] + np.asarray(centre, dtype=np.float64)
    if order == "morton":
        pts = pts[morton_order(pts)]
    return np.ascontiguousarray(pts)


def box_surface(lo, hi, n: int = 1, q: int = 1) -> np.ndarray:
    """Outward-oriented axis-aligned box [lo,hi] as 6*n*n order-q faces (used by
    tests for flat and concave geometry)."""
    P = cube_face_points(n, q).astype(np.float64) / (n * q)  # in [-1, 1]
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return np.ascontiguousarray(0.5 * (lo + hi) + 0.5 * (hi - lo) * P)


# --------------------------------------------------------------------------
# the named workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass
class CutCase:
    name: str
    p: int
    n: int
    nodes: np.ndarray          # [n_elem][(p+1)^3][3]
    q: int
    faces: np.ndarray          # [n_faces][(q+1)^2][3]
    pose: np.ndarray | None = None  # 3x4 [R|t] applied to faces, or None
    centre: np.ndarray | None = None  # centre of the (sphere-like) surface, before the pose

    @property
    def n_elem(self) -> int:
        return self.nodes.shape[0]

    @property
    def n_faces(self) -> int:
        return self.faces.shape[0]


def sphere_in_box(n: int = 16, p: int = 2, m: int = 8, q: int = 2, seed: int = 1, jitter: float = 0.05,
                  offset: float = 0.1, radius: float = 1.0) -> CutCase:
    """Background n^3 order-p hexes on [-2,2]^3 with node jitter +-jitter*h; cut
    surface a cubed sphere of the given radius, 6*m*m order-q faces, centred at
    a seeded offset in [-offset, offset]^3.  n=16,p=2,m=8,q=2 is the 4096-element
    plain workload."""
    g = rng(seed)
    centre = g.uniform(-offset, offset, size=3)
    nodes = background(n, p, jitter=jitter, seed=seed + 1000)
    faces = cubed_sphere(m, q, radius=radius, centre=centre)
    return CutCase(f"sphere{n}^3Q{p}_m{m}q{q}", p, n, nodes, q, faces, centre=centre)


def dimpled_sphere_case(n: int = 64, p: int = 2, m: int = 32, q: int = 2, seed: int = 2, n_dimples: int = 336,
                        sinusoid: float = 0.1, offset: float = 0.1) -> CutCase:
    """Background n^3 order-p hexes on [-2,2]^3 curved by a sinusoidal node
    displacement of amplitude sinusoid*h; cut surface a dimpled sphere
    r = 1 - 0.01*sum Gaussian dimples (width 0.08) at a randomly rotated
    Fibonacci lattice of ``n_dimples`` centres, 6*m*m order-q faces.
    n=64,p=2,m=32,q=2 is the 262,144-element scale workload."""
    g = rng(seed)
    rot = random_rotation(g)
    centre = g.uniform(-offset, offset, size=3)
    centres = fibonacci_sphere(n_dimples, rot)
    nodes = background(n, p, sinusoid=sinusoid)
    faces = cubed_sphere(m, q, radius=1.0, centre=centre, dimples=centres)
    return CutCase(f"dimpled{n}^3Q{p}_m{m}q{q}", p, n, nodes, q, faces, centre=centre)


def batch_cases(count: int = 256, seed: int = 3, n_range=(8, 40), m_choices=(8, 16, 24, 32), p: int = 2,
                q: int = 2, jitter: float = 0.05):
    """Independent instances: background n^3 order-p hexes with n uniform in
    n_range, cubed sphere 6*m*m order-q faces with m drawn from m_choices,
    random rotation and an offset in [-0.1,0.1]^3 per instance.  Returns the
    list of CutCases (each sphere given through its pose)."""
    g = rng(seed)
    out = []
    base_faces = {}
    for i in range(count):
        n = int(g.integers(n_range[0], n_range[1] + 1))
        m = int(m_choices[int(g.integers(0, len(m_choices)))])
        rot = random_rotation(g)
        off = g.uniform(-0.1, 0.1, size=3)
        if m not in base_faces:
            base_faces[m] = cubed_sphere(m, q)
        pose = np.concatenate([rot, off.reshape(3, 1)], axis=1)
        nodes = background(n, p, jitter=jitter, seed=seed * 100003 + i)
        out.append(CutCase(f"batch{i}_{n}^3_m{m}", p, n, nodes, q, base_faces[m], pose, np.zeros(3)))
    return out


def polycube_surface(cells, scale: float = 1.0, origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Outward-oriented, watertight boundary of a union of unit lattice cubes
    (``cells`` = iterable of integer (x, y, z)): one order-1 face per cube face
    that separates an occupied cell from an empty one.  Used for slot, groove
    and concave-corner surfaces."""
    occ = {tuple(int(v) for v in c) for c in cells}
    faces = []
    for c in sorted(occ):
        for ax, sg, axi, aeta in _CUBE_FACES:
            nb = list(c)
            nb[ax] += sg
            if tuple(nb) in occ:
                continue
            quad = np.zeros((4, 3), dtype=np.float64)
            for j in range(2):
                for i in range(2):
                    pt = [float(v) for v in c]
                    pt[ax] += 1.0 if sg > 0 else 0.0
                    pt[axi] += float(i)
                    pt[aeta] += float(j)
                    quad[i + 2 * j] = pt
            faces.append(quad)
    F = np.stack(faces)
    return np.ascontiguousarray(np.asarray(origin, dtype=np.float64) + scale * F)


def hex_block(lo, hi, p: int = 1, n=(1, 1, 1)) -> np.ndarray:
    """An axis-aligned block [lo,hi] split into n[0] x n[1] x n[2] order-p hexes
    (straight-sided), node layout as ``background``."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    out = []
    for ez in range(n[2]):
        for ey in range(n[1]):
            for ex in range(n[0]):
                e0 = lo + (hi - lo) * np.array([ex, ey, ez]) / np.array(n)
                e1 = lo + (hi - lo) * np.array([ex + 1, ey + 1, ez + 1]) / np.array(n)
                nodes = np.zeros(((p + 1) ** 3, 3))
                for k in range(p + 1):
                    for j in range(p + 1):
                        for i in range(p + 1):
                            t = np.array([i, j, k], dtype=np.float64) / p
                            nodes[i + (p + 1) * (j + (p + 1) * k)] = e0 + (e1 - e0) * t
                out.append(nodes)
    return np.ascontiguousarray(np.stack(out))
