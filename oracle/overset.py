"""Set logic after the cut: the union of several cuts, artificial-boundary
faces, and the unblank procedure of a moving grid (plain Python/numpy).

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: imported by the test suite
and nothing else; the CUDA library shares no code with it.

Readings (the paper states these steps in words only):
* blanked by one cut (Sec. 4.2, final paragraphs; Sec. 2 on hole cutting):
  an element inside the surface (HOLE) is removed; an element the surface
  passes through (FRINGE, distance <= tol) is kept when the surface is an
  overset boundary (the element is needed for overlap) and removed when it is
  a solid wall (no computed element may reach inside the body);
* union (Sec. 4.2, last paragraph): an element is removed when any cut
  removes it;
* artificial-boundary faces (Sec. 4.2, last paragraph): faces with a removed
  element on one side and a kept element on the other, reported on the kept
  side (that element's flux points receive interpolated data);
* unblank (Algorithm "Artificial Boundary unblank procedure", Sec. 3): with
  I_t- the removal state of the previous step and the cuts at t and t + dt,
  wall cuts remove what either cut removes ("any cell which becomes a hole in
  I_t+ can be set to hole in I_t"); overset cuts remove only what both remove
  (cells are not blanked until they are no longer needed); an element removed
  in I_t- and kept now must be unblanked.
"""
from __future__ import annotations

import numpy as np

HOLE, FIELD, FRINGE = 0, 1, -1
WALL, OVERSET = 0, 1


def removed(flags, kind):
    """Elements one cut removes: HOLE, and FRINGE too for a wall cut."""
    f = np.asarray(flags)
    return (f == HOLE) | ((f == FRINGE) if kind == WALL else np.zeros(f.shape, dtype=bool))


def union(flag_sets, kinds):
    """Removal after several cuts: removed by any of them."""
    out = np.zeros(np.asarray(flag_sets[0]).shape, dtype=bool)
    for f, k in zip(flag_sets, kinds):
        out |= removed(f, k)
    return out


def ab_faces(rem, neighbours):
    """Per element a 6-bit mask: bit j set when the element is kept and its
    neighbour across local face j (-1: none) is removed.  Faces 0..5 are
    xi = -1, +1, eta = -1, +1, zeta = -1, +1."""
    rem = np.asarray(rem, dtype=bool)
    nb = np.asarray(neighbours)
    mask = np.zeros(rem.shape[0], dtype=np.uint8)
    for e in range(rem.shape[0]):
        if rem[e]:
            continue
        for j in range(6):
            o = nb[e, j]
            if o >= 0 and rem[o]:
                mask[e] |= np.uint8(1 << j)
    return mask


def unblank(prev_removed, flags_t, flags_tp, kind):
    """(removed now, to unblank) for one cut kind: wall removes what the cut at
    t or at t + dt removes, overset what both remove; an element removed
    before and kept now is unblanked."""
    rt, rtp = removed(flags_t, kind), removed(flags_tp, kind)
    now = (rt | rtp) if kind == WALL else (rt & rtp)
    prev = np.asarray(prev_removed, dtype=bool)
    return now, prev & ~now


def structured_neighbours(nx, ny, nz):
    """Face neighbours of the hexes of an nx*ny*nz block numbered
    ex + nx*(ey + ny*ez): [n][6] in face order xi-, xi+, eta-, eta+, zeta-,
    zeta+, -1 on the block boundary."""
    n = nx * ny * nz
    out = np.full((n, 6), -1, dtype=np.int64)
    for ez in range(nz):
        for ey in range(ny):
            for ex in range(nx):
                e = ex + nx * (ey + ny * ez)
                if ex > 0: out[e, 0] = e - 1
                if ex < nx - 1: out[e, 1] = e + 1
                if ey > 0: out[e, 2] = e - nx
                if ey < ny - 1: out[e, 3] = e + nx
                if ez > 0: out[e, 4] = e - nx * ny
                if ez < nz - 1: out[e, 5] = e + nx * ny
    return out
