"""The closed form that spares the oracle the elements far from a sphere-like
surface (tests/sphere_split.py) gives the oracle's own flags wherever it
decides, on every element of small cases -- plain, dimpled, jittered, posed."""
import numpy as np

import oracle as O
import sphere_split as SS
import workloads as W


def _check(case, pose=None):
    full, _, _, st = O.cut(case.p, case.nodes, case.q, case.faces, pose=pose)
    assert st["undecidable"] == 0
    got, n_oracle = SS.expected_flags(O, case.p, case.nodes, case.q, case.faces, case.centre, pose=pose)
    assert np.array_equal(got, full)
    # the closed form really decides most elements (else it would test nothing)
    assert n_oracle < 0.6 * case.n_elem
    return n_oracle


def test_plain_sphere_in_jittered_box():
    _check(W.sphere_in_box(n=12, p=2, m=6, q=2, seed=1))


def test_dimpled_sphere_curved_grid():
    _check(W.dimpled_sphere_case(n=12, m=8, n_dimples=40, seed=5))


def test_posed_batch_instances():
    for cs in W.batch_cases(count=3, seed=21, n_range=(10, 12), m_choices=(8,)):
        _check(cs, pose=cs.pose)


def test_split_puts_every_straddling_element_in_the_rest():
    # a sphere of radius 1 about the origin and a 1/8-spaced lattice: an
    # element with nodes on both sides of r = 1 is never classified by the
    # closed form
    nodes = W.background(16, 1)
    r = np.sqrt((nodes ** 2).sum(axis=2))
    hole, field, rest = SS.split(nodes, np.zeros(3), 0.999, 1.0)
    both = np.nonzero((r.min(axis=1) < 1.0) & (r.max(axis=1) > 1.0))[0]
    assert np.isin(both, rest).all()
    assert np.intersect1d(hole, field).size == 0
    assert hole.size + field.size + rest.size == nodes.shape[0]
