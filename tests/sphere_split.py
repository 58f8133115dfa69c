"""Element-by-element expected flags for a cut by a sphere-like surface, without
running the oracle on elements far from it.

For a closed surface S around a centre c, let r_in be the smallest distance
from c to S's triangles (the oracle's point-surface distance) and r_out the
largest distance from c to a face node (every surface triangle lies in the
convex hull of its nodes, so within r_out of c).  For an element E:

* every boundary triangle of E lies in the convex hull of E's nodes, hence in
  the ball of radius max_node |x - c|.  If that radius is below r_in - margin,
  E is farther than tol from S and lies in the component of c: HOLE, provided
  c itself is inside S (winding number 1, checked with the oracle).
* every point of a boundary triangle of E lies within the diagonal of E's node
  box of one of E's nodes, so at least min_node |x - c| - diag from c.  If that
  exceeds r_out + margin, E is farther than tol from S and lies in the
  unbounded component: FIELD.

Every other element goes to the oracle.  The margin (1e-6) is ten times tol and
far above any rounding of these distances.
"""
from __future__ import annotations

import numpy as np

MARGIN = 1e-6


def split(nodes: np.ndarray, centre, r_in: float, r_out: float):
    """(hole, field, rest) index arrays of the elements."""
    c = np.asarray(centre, dtype=np.float64)
    hole, field, rest = [], [], []
    for s in range(0, nodes.shape[0], 1 << 16):
        X = nodes[s:s + (1 << 16)]
        r = np.sqrt(((X - c) ** 2).sum(axis=2))
        diag = np.sqrt(((X.max(axis=1) - X.min(axis=1)) ** 2).sum(axis=1))
        h = r.max(axis=1) < r_in - MARGIN
        f = r.min(axis=1) - diag > r_out + MARGIN
        idx = np.arange(s, s + X.shape[0])
        hole.append(idx[h])
        field.append(idx[f])
        rest.append(idx[~h & ~f])
    return np.concatenate(hole), np.concatenate(field), np.concatenate(rest)


def surface_radii(O, q: int, posed_faces: np.ndarray, centre):
    """(r_in, r_out, winding number at the centre) of a posed surface."""
    c = np.asarray(centre, dtype=np.float64)
    tris = O.surface_tris(q, posed_faces)
    r_in, w = O.point_surface(c, tris)
    r_out = float(np.sqrt(((posed_faces.reshape(-1, 3) - c) ** 2).sum(axis=1)).max())
    return float(r_in), r_out, float(w)


def expected_flags(O, p: int, nodes: np.ndarray, q: int, faces: np.ndarray, centre, pose=None, nthreads=0):
    """Flags of every element: closed form away from the surface, the oracle
    near it.  ``centre`` is the surface's centre before the pose.  Returns
    (flags, number of elements the oracle classified)."""
    posed = O.apply_pose(faces, pose)
    c = np.asarray(centre, dtype=np.float64)
    if pose is not None:
        P = np.asarray(pose, dtype=np.float64).reshape(3, 4)
        c = P[:, :3] @ c + P[:, 3]
    r_in, r_out, w = surface_radii(O, q, posed, c)
    assert abs(w - 1.0) < 1e-6, f"the centre is not inside the surface (winding number {w})"
    hole, field, rest = split(nodes, c, r_in, r_out)
    flags = np.full(nodes.shape[0], 9, dtype=np.int8)
    flags[hole] = O.HOLE
    flags[field] = O.FIELD
    if rest.size:
        rf, _, _, st = O.cut(p, nodes, q, faces, pose=pose, ids=rest, nthreads=nthreads)
        assert st["undecidable"] == 0
        flags[rest] = rf
    return flags, int(rest.size)
