"""Pins of the oracle's element-face distance d(E, F) (oracle.pair_dist), the
per-pair quantity behind the grazing fraction of the precision-stress
workload: a closed form, the definition taken through the separately pinned
triangle routines, and consistency with the cut's own element distance."""
import numpy as np

import oracle as O
import workloads as W


def test_axis_aligned_gap_is_the_distance():
    # unit cube element [0,1]^3 (p = 1, 2) and a flat square face in the plane
    # x = 1 + g over [0.25, 0.75]^2: the distance is the gap g
    for p in (1, 2):
        el = W.hex_block([0, 0, 0], [1, 1, 1], p=p)
        for g in (0.0, 2.0 ** -30, 0.125, 3.0):  # 1 + g exact in FP64
            face = np.array([[[1 + g, 0.25, 0.25], [1 + g, 0.75, 0.25], [1 + g, 0.25, 0.75], [1 + g, 0.75, 0.75]]])
            d = O.pair_dist(p, el, 1, face, [0], [0])
            assert d[0] == g


def test_definition_through_the_triangle_routines():
    c = W.dimpled_sphere_case(n=6, m=3, n_dimples=12, seed=9)
    g = np.random.default_rng(2)
    es = g.choice(c.n_elem, 6, replace=False)
    fs = g.choice(c.n_faces, 6, replace=False)
    got = O.pair_dist(c.p, c.nodes, c.q, c.faces, es, fs)
    for k, (e, f) in enumerate(zip(es, fs)):
        et = O.elem_tris(c.p, c.nodes[e])
        ft = O.face_tris(c.q, c.faces[f])
        want = min(O.tritri(a, b)[0] for a in et for b in ft)
        assert got[k] == want


def test_element_distance_is_the_minimum_over_faces():
    c = W.sphere_in_box(n=8, p=2, m=4, q=2, seed=3)
    pose = np.concatenate([W.random_rotation(W.rng(7)), np.array([[0.03], [-0.02], [0.01]])], axis=1)
    posed = O.apply_pose(c.faces, pose)
    ids = np.arange(0, c.n_elem, 37)
    _, dist, _, _ = O.cut(c.p, c.nodes, c.q, c.faces, pose=pose, ids=ids)
    E = np.repeat(ids, c.n_faces)
    F = np.tile(np.arange(c.n_faces), ids.size)
    d = O.pair_dist(c.p, c.nodes, c.q, posed, E, F).reshape(ids.size, c.n_faces)
    assert np.array_equal(d.min(axis=1), np.abs(dist))
