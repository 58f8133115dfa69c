"""Pins for the oracle's element classification (Sec. 4.2 of the paper:
every element computes its signed minimum distance to the cut surface and is
hole, fringe ("intersecting") or field from it).

Pins used, none of which re-types the oracle's own code:
  * brute force over all faces == branch-and-bound over faces,
  * closed form for a sphere in an unjittered box (inscribed / circumscribed
    balls bound every element),
  * invariants (fringe separates hole from field; nested spheres give nested
    holes; hole/fringe counts bracket the enclosed volume),
  * dense point sampling of each element's boundary on tiny meshes,
  * the paper's own side rule agreeing with the winding number, including the
    slot and concave-corner geometries of Sec. 4.1 / 5 (equidistant faces),
  * closed forms for the solid-angle winding number and the linearisation.
"""
import itertools

import numpy as np
import pytest

import oracle as O
import workloads as W

HOLE, FIELD, FRINGE = O.HOLE, O.FIELD, O.FRINGE


# --------------------------------------------------------------- linearisation
def _my_elem_tris(p, nodes):
    """Independent restatement of the element boundary triangulation reading:
    each of the 6 faces is a (p+1)^2 node grid, each grid quad split along its
    (00)-(11) diagonal."""
    idx = lambda i, j, k: i + (p + 1) * (j + (p + 1) * k)
    out = set()
    for fix_axis in range(3):
        for fix in (0, p):
            for a in range(p):
                for b in range(p):
                    def nd(u, v):
                        ijk = [None, None, None]
                        free = [ax for ax in range(3) if ax != fix_axis]
                        ijk[fix_axis] = fix
                        ijk[free[0]] = u
                        ijk[free[1]] = v
                        return idx(*ijk)
                    q00, q10, q11, q01 = nd(a, b), nd(a + 1, b), nd(a + 1, b + 1), nd(a, b + 1)
                    for tri in ((q00, q10, q11), (q00, q11, q01)):
                        out.add(frozenset(tuple(nodes[t]) for t in tri))
    return out


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_element_triangulation(p):
    nodes = W.background(1, p, jitter=0.05, seed=p)[0]
    T = O.elem_tris(p, nodes)
    assert T.shape == (12 * p * p, 3, 3)
    got = {frozenset(tuple(v) for v in t) for t in T}
    assert got == _my_elem_tris(p, nodes)
    # watertight: every edge shared by exactly two triangles
    edges = {}
    for t in T:
        for i in range(3):
            e = frozenset((tuple(t[i]), tuple(t[(i + 1) % 3])))
            edges[e] = edges.get(e, 0) + 1
    assert set(edges.values()) == {2}


def test_face_triangulation_orientation_and_volume():
    F = W.cubed_sphere(6, 2)
    T = O.surface_tris(2, F)
    # closed + outward: signed volume positive and close to the ball volume
    v = O.signed_volume(T)
    assert 0.95 * 4 / 3 * np.pi < v < 4 / 3 * np.pi
    edges = {}
    for t in T:
        for i in range(3):
            e = (tuple(t[i]), tuple(t[(i + 1) % 3]))
            edges[e] = edges.get(e, 0) + 1
    # consistently oriented closed surface: each directed edge once, reversed once
    for (a, b), c in edges.items():
        assert c == 1 and edges.get((b, a)) == 1


# --------------------------------------------------------------- winding number
def test_winding_closed_forms():
    # the octant triangle subtends pi/2 steradian from the origin: w = 1/8
    T = np.array([[[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]]])
    assert O.winding([0, 0, 0], T) == pytest.approx(0.125, rel=1e-14)
    # a polycube of 5 cells: unit winding inside, zero outside, volume 5
    cells = [(0, 0, 0), (1, 0, 0), (2, 0, 0), (0, 1, 0), (2, 1, 0)]
    S = O.surface_tris(1, W.polycube_surface(cells))
    assert O.signed_volume(S) == pytest.approx(5.0, rel=1e-14)
    for c in cells:
        assert O.winding(np.array(c) + 0.5, S) == pytest.approx(1.0, abs=1e-12)
    for pt in ([1.5, 1.5, 0.5], [-0.5, 0.5, 0.5], [1.0, 0.5, 3.0]):
        assert O.winding(pt, S) == pytest.approx(0.0, abs=1e-12)


def test_pose_transform():
    F = W.cubed_sphere(2, 2)
    # quarter turn about z plus a dyadic shift: exact in floating point
    pose = np.array([[0.0, -1.0, 0.0, 0.5], [1.0, 0.0, 0.0, -0.25], [0.0, 0.0, 1.0, 2.0]])
    G = O.apply_pose(F, pose)
    assert np.array_equal(G[..., 0], -F[..., 1] + 0.5)
    assert np.array_equal(G[..., 1], F[..., 0] - 0.25)
    assert np.array_equal(G[..., 2], F[..., 2] + 2.0)


# --------------------------------------------------------------- brute == pruned
@pytest.mark.parametrize("n,p,m,q,jit", [(6, 1, 3, 1, 0.05), (6, 2, 3, 2, 0.05), (5, 3, 2, 3, 0.0), (4, 4, 2, 2, 0.1)])
def test_pruned_equals_brute(n, p, m, q, jit):
    c = W.sphere_in_box(n=n, p=p, m=m, q=q, jitter=jit, seed=7 + n)
    f1, d1, pf1, s1 = O.cut(p, c.nodes, q, c.faces, brute=True)
    f2, d2, pf2, s2 = O.cut(p, c.nodes, q, c.faces, brute=False)
    assert np.array_equal(f1, f2) and np.array_equal(pf1, pf2)
    assert np.array_equal(d1, d2)
    assert s1["undecidable"] == 0 and s1["paper_rule_disagree"] == 0
    assert s2["tritri_tests"] < s1["tritri_tests"]
    assert s1["fringe"] > 0 and s1["field"] > 0


def test_pruned_equals_brute_dimpled_and_posed():
    c = W.dimpled_sphere_case(n=6, p=2, m=4, q=2, n_dimples=24)
    pose = np.concatenate([W.random_rotation(W.rng(5)), np.array([[0.05], [-0.02], [0.07]])], axis=1)
    f1, d1, _, s1 = O.cut(2, c.nodes, 2, c.faces, pose=pose, brute=True)
    f2, d2, _, s2 = O.cut(2, c.nodes, 2, c.faces, pose=pose)
    assert np.array_equal(f1, f2) and np.array_equal(d1, d2)
    # the pose is the same as handing the oracle pre-transformed faces
    f3, d3, _, _ = O.cut(2, c.nodes, 2, O.apply_pose(c.faces, pose))
    assert np.array_equal(f1, f3) and np.array_equal(d1, d3)


# --------------------------------------------------------------- closed form
@pytest.mark.parametrize("n,p,m", [(8, 1, 6), (10, 2, 6), (8, 3, 4)])
def test_sphere_in_unjittered_box_closed_form(n, p, m):
    R = 1.0
    c = W.sphere_in_box(n=n, p=p, m=m, q=2, jitter=0.0, offset=0.1, seed=11 + n)
    centre = W.rng(11 + n).uniform(-0.1, 0.1, size=3)  # the generator's centre
    flags, dist, pflags, st = O.cut(p, c.nodes, 2, c.faces)
    S = O.surface_tris(2, c.faces)
    # radius of a ball about the centre free of surface points: min plane distance
    nrm = np.cross(S[:, 1] - S[:, 0], S[:, 2] - S[:, 0])
    r_in = np.min(np.abs(np.einsum("ij,ij->i", nrm, S[:, 0] - centre)) / np.linalg.norm(nrm, axis=1))
    tol = 1e-7
    n_hole_claims = n_field_claims = 0
    for e in range(c.n_elem):
        X = c.nodes[e]
        rmax = np.max(np.linalg.norm(X - centre, axis=1))
        lo, hi = X.min(axis=0), X.max(axis=0)
        boxd = np.linalg.norm(np.maximum(0.0, np.maximum(lo - centre, centre - hi)))
        if rmax < r_in - tol:
            assert flags[e] == HOLE, e
            assert -dist[e] >= r_in - rmax - 1e-12
            n_hole_claims += 1
        elif boxd > R + tol:
            assert flags[e] == FIELD, e
            assert dist[e] >= boxd - R - 1e-12
            n_field_claims += 1
    assert n_hole_claims > 0 and n_field_claims > 0
    assert st["undecidable"] == 0 and st["paper_rule_disagree"] == 0


# --------------------------------------------------------------- invariants
def _grid_flags(flags, n):
    return flags.reshape(n, n, n)  # [ez][ey][ex]


@pytest.mark.parametrize("case", ["sphere", "dimpled"])
def test_fringe_separates_hole_from_field(case):
    if case == "sphere":
        c = W.sphere_in_box(n=16, p=2, m=8, q=2)
    else:
        c = W.dimpled_sphere_case(n=12, p=2, m=8, q=2, n_dimples=60)
    flags, dist, pflags, st = O.cut(c.p, c.nodes, c.q, c.faces)
    G = _grid_flags(flags, c.n)
    for ax in range(3):
        a = np.moveaxis(G, ax, 0)
        pair = {(int(x), int(y)) for x, y in zip(a[:-1].ravel(), a[1:].ravel())}
        assert (HOLE, FIELD) not in pair and (FIELD, HOLE) not in pair
    assert np.all((flags == FRINGE) == (np.abs(dist) <= 1e-7))
    assert np.all(dist[flags == HOLE] < 0) and np.all(dist[flags == FIELD] > 0)
    # the hole is enclosed: no hole element on the grid boundary
    assert not np.any(G[[0, -1]] == HOLE) and not np.any(G[:, [0, -1]] == HOLE) and not np.any(G[:, :, [0, -1]] == HOLE)
    assert st["paper_rule_disagree"] == 0 and st["undecidable"] == 0


def test_nested_spheres_and_volume_bracket():
    n, p = 12, 1
    nodes = W.background(n, p)
    h = 4.0 / n
    prev_hole = None
    for R in (0.6, 0.9, 1.2):
        F = W.cubed_sphere(8, 2, radius=R, centre=(0.031, -0.017, 0.023))
        flags, dist, _, st = O.cut(p, nodes, 2, F)
        vol = O.signed_volume(O.surface_tris(2, F))
        nh, nf = np.sum(flags == HOLE), np.sum(flags == FRINGE)
        assert nh * h ** 3 <= vol <= (nh + nf) * h ** 3
        hole = flags == HOLE
        if prev_hole is not None:
            assert np.all(hole[prev_hole])
        prev_hole = hole
        assert st["paper_rule_disagree"] == 0


# --------------------------------------------------------------- dense sampling
def _boundary_samples(p, nodes, k):
    T = O.elem_tris(p, nodes)
    pts = []
    for t in T:
        for i in range(k + 1):
            for j in range(k + 1 - i):
                pts.append(t[0] + (i / k) * (t[1] - t[0]) + (j / k) * (t[2] - t[0]))
    longest = max(np.linalg.norm(t[a] - t[b]) for t in T for a, b in ((0, 1), (1, 2), (2, 0)))
    return np.array(pts), longest / k


@pytest.mark.parametrize("n,p,q,R", [(3, 1, 1, 0.8), (3, 2, 2, 0.7), (4, 1, 2, 1.05)])
def test_dense_point_sampling(n, p, q, R):
    nodes = W.background(n, p, jitter=0.08, seed=3 * n + p, lo=-1.5, hi=1.5)
    F = W.cubed_sphere(3, q, radius=R, centre=(0.04, -0.03, 0.02))
    S = O.surface_tris(q, F)
    flags, dist, _, st = O.cut(p, nodes, q, F)
    tol = 1e-7
    for e in range(nodes.shape[0]):
        P, gap = _boundary_samples(p, nodes[e], 5)
        ds, ws = zip(*(O.point_surface(x, S) for x in P))
        ds, ws = np.array(ds), np.array(ws)
        d = abs(dist[e])
        assert d <= ds.min() + 1e-14
        assert d >= ds.min() - gap
        sides = set((ws > 0.5).tolist())
        if len(sides) == 2:
            assert flags[e] == FRINGE
        if ds.min() - gap > tol:
            assert flags[e] != FRINGE
            assert flags[e] == (HOLE if ws[0] > 0.5 else FIELD)
    assert st["paper_rule_disagree"] == 0


# --------------------------------------------------------------- slot / corner
def test_slot_equidistant_faces_keep_the_larger_dot():
    # U-shaped block (Sec. 5 slot geometry): cells x in 0..2, y in 0..1, with the
    # slot at x=1, y=1 open towards +y; elements sit centred in the slot.
    cells = [(x, y, z) for x in range(3) for y in range(2) for z in range(2) if not (x == 1 and y == 1)]
    F = W.polycube_surface(cells)
    # 1x1 slot cross-section; elements of size 0.5 centred in it, equidistant
    # from the two slot walls
    elems = W.hex_block([1.25, 1.25, 0.25], [1.75, 1.75, 1.75], p=1, n=(1, 1, 3))
    inside = W.hex_block([0.25, 0.25, 0.25], [0.75, 0.75, 0.75], p=2)
    far = W.hex_block([4.0, 4.0, 4.0], [4.5, 4.5, 4.5], p=1)
    nodes = np.concatenate([elems, W.hex_block([0.25, 0.25, 0.25], [0.75, 0.75, 0.75], p=1), far])
    flags, dist, pflags, st = O.cut(1, nodes, 1, F)
    assert list(flags[:3]) == [FIELD, FIELD, FIELD]
    assert list(pflags[:3]) == [FIELD, FIELD, FIELD]
    assert flags[3] == HOLE and pflags[3] == HOLE
    assert flags[4] == FIELD
    assert np.allclose(dist[:3], 0.25)
    assert st["paper_rule_disagree"] == 0 and st["undecidable"] == 0
    f2, _, p2, _ = O.cut(2, inside, 1, F)
    assert f2[0] == HOLE and p2[0] == HOLE


def test_concave_corner():
    # L-shaped block: the reflex edge at (1,1,z); an element in the notch is
    # equidistant from the two faces meeting there (Fig. multinorm (b))
    cells = [(0, 0, 0), (1, 0, 0), (0, 1, 0)]
    F = W.polycube_surface(cells)
    notch = W.hex_block([1.2, 1.2, 0.3], [1.6, 1.6, 0.7], p=1)
    corner_out = W.hex_block([2.2, 2.2, 0.3], [2.4, 2.4, 0.5], p=1)  # beyond the convex corner
    pocket_in = W.hex_block([0.6, 0.6, 0.3], [0.9, 0.9, 0.6], p=2)
    flags, dist, pflags, st = O.cut(1, np.concatenate([notch, corner_out]), 1, F)
    assert list(flags) == [FIELD, FIELD] and list(pflags) == [FIELD, FIELD]
    assert dist[0] == pytest.approx(0.2, rel=1e-12)
    f2, d2, p2, _ = O.cut(2, pocket_in, 1, F)
    assert f2[0] == HOLE and p2[0] == HOLE
    assert d2[0] == pytest.approx(-0.1 * np.sqrt(2.0), rel=1e-12)  # nearest: the reflex edge


def test_intersecting_element_is_fringe_with_zero_distance():
    F = W.polycube_surface([(0, 0, 0)])
    e = W.hex_block([0.5, 0.5, 0.5], [1.5, 1.5, 1.5], p=2)
    flags, dist, _, _ = O.cut(2, e, 1, F)
    assert flags[0] == FRINGE and dist[0] == 0.0
    # an element touching the surface within tol is fringe too
    e2 = W.hex_block([1.0 + 5e-8, 0.2, 0.2], [1.5, 0.8, 0.8], p=1)
    flags, dist, _, _ = O.cut(1, e2, 1, F)
    assert flags[0] == FRINGE and dist[0] == pytest.approx(5e-8, rel=1e-6)
    e3 = W.hex_block([1.0 + 5e-7, 0.2, 0.2], [1.5, 0.8, 0.8], p=1)
    flags, dist, _, _ = O.cut(1, e3, 1, F)
    assert flags[0] == FIELD
