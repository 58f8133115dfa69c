"""The stored necessary pair sets (tests/golden/necessary_pairs.json) are what
the oracle counts today, and the set of elements they cover holds every
element the full oracle cut finds within tol of the surface."""
import importlib.util
import json
import os

import numpy as np
import pytest

import oracle as O

pytest.importorskip("scipy")
HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location("necessary_pairs", os.path.join(HERE, "golden", "necessary_pairs.py"))
NP = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(NP)
STORED = json.load(open(os.path.join(HERE, "golden", "necessary_pairs.json")))


@pytest.mark.parametrize("name", ["plain16", "mid32", "scale64"])
def test_stored_counts_reproduce(name):
    got = NP.count(NP.workloads()[name]())
    assert got == STORED[name]


def test_exact_test_elements_hold_every_fringe_element():
    case = NP.workloads()["plain16"]()
    flags, dist, _, _ = O.cut(case.p, case.nodes, case.q, case.faces)
    ids = NP.exact_test_elements(case.nodes, case.faces)
    fringe = np.nonzero(flags == O.FRINGE)[0]
    assert np.isin(fringe, ids).all()
    assert fringe.size == STORED["plain16"]["fringe"]
    # outside the set every element is farther than tol: its box already is
    rest = np.setdiff1d(np.arange(case.n_elem), ids)
    assert np.all(np.abs(dist[rest]) > NP.TOL)


def test_necessary_set_is_a_lower_bound_of_brute_force_work():
    """On a few elements of the plain workload, S* is contained in what the
    brute-force oracle visits, and it is not empty for a fringe element."""
    case = NP.workloads()["plain16"]()
    ids = NP.exact_test_elements(case.nodes, case.faces)[:12]
    _, _, _, pr = O.cut(case.p, case.nodes, case.q, case.faces, ids=ids)
    _, _, _, br = O.cut(case.p, case.nodes, case.q, case.faces, ids=ids, brute=True)
    assert pr["s_star_pairs"] == br["s_star_pairs"] > 0
    assert pr["s_star_tri_pairs"] == br["s_star_tri_pairs"]
    nte, ntf = 12 * case.p ** 2, 2 * case.q ** 2
    assert br["tritri_tests"] == ids.size * case.n_faces * nte * ntf
    assert pr["s_star_tri_pairs"] <= pr["s_star_pairs"] * nte * ntf <= br["tritri_tests"]
