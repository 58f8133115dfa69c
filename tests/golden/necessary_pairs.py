"""Writes necessary_pairs.json: the necessary pair set S* of each benchmark
workload, counted by the oracle.

The exact test (Sec. 4.2, the curved element-face test) has to be run on an
element E when no bounding-box test can clear it: when E's box lies within tol
of some face box.  For such an element, any method that prunes by boxes and
returns the exact minimum distance d(E) must evaluate every face F whose box
lies within d(E) of E's box:

    S*(E) = { F : boxdist(E, F) <= d(E) }.

The oracle computes d(E) and counts S*(E) (element-face pairs) and the
triangle pairs of S* whose triangle boxes lie within d(E).  The algorithmic
work of the exact test is |S*| x n_Tc x n_T(F) x C_tt, with n_Tc = 3 x 2p^2 (the
element triangles on the three faces at the nearest corner that the paper's
second pass visits) as the lower count and 12p^2 (all six faces) as the upper
one, n_T(F) = 2q^2 face triangles, and C_tt the arithmetic of one
triangle-triangle distance.

Calls only the oracle and the seeded input generators.  Run from the
repository root:  python tests/golden/necessary_pairs.py
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "necessary_pairs.json")
TOL = 1e-7


def workloads():
    sys.path.insert(0, ROOT)
    import workloads as W
    return {
        "scale64": W.dimpled_sphere_case,
        "mid32": lambda: W.dimpled_sphere_case(n=32, m=16, seed=12),
        "plain16": lambda: W.sphere_in_box(n=16, p=2, m=8, q=2, seed=1),
    }


def exact_test_elements(nodes: np.ndarray, faces: np.ndarray, tol: float = TOL) -> np.ndarray:
    """Elements whose node box lies within tol of some face node box, ascending."""
    from scipy.spatial import cKDTree
    eb = np.concatenate([nodes.min(1), nodes.max(1)], 1)
    fb = np.concatenate([faces.min(1), faces.max(1)], 1)
    ec = 0.5 * (eb[:, :3] + eb[:, 3:])
    fc = 0.5 * (fb[:, :3] + fb[:, 3:])
    re = 0.5 * np.linalg.norm(eb[:, 3:] - eb[:, :3], axis=1).max()
    rf = 0.5 * np.linalg.norm(fb[:, 3:] - fb[:, :3], axis=1).max()
    # every pair of boxes within tol has centres within re + rf + tol
    lists = cKDTree(ec).query_ball_point(fc, re + rf + 2 * tol)
    hit = np.zeros(nodes.shape[0], dtype=bool)
    for f, L in enumerate(lists):
        if not L:
            continue
        L = np.asarray(L, dtype=np.int64)
        gap = np.maximum(0.0, np.maximum(eb[L, :3] - fb[f, 3:], fb[f, :3] - eb[L, 3:]))
        hit[L[np.sqrt((gap * gap).sum(1)) <= tol]] = True
    return np.nonzero(hit)[0]


def count(case) -> dict:
    sys.path.insert(0, ROOT)
    import oracle as O
    ids = exact_test_elements(case.nodes, case.faces)
    flags, _, _, st = O.cut(case.p, case.nodes, case.q, case.faces, ids=ids)
    return {
        "n_elem": int(case.n_elem), "n_faces": int(case.n_faces), "p": int(case.p), "q": int(case.q),
        "tol": TOL,
        "exact_test_elements": int(ids.size),
        "fringe": int((flags == O.FRINGE).sum()),
        "s_star_pairs": int(st["s_star_pairs"]),
        "s_star_tri_pairs": int(st["s_star_tri_pairs"]),
        "n_tc_lower": 3 * 2 * case.p * case.p,
        "n_tc_upper": 12 * case.p * case.p,
        "n_tf": 2 * case.q * case.q,
    }


def main():
    out = {"definition": "S*(E) = {F : boxdist(E,F) <= d(E)} over the elements whose box lies within tol "
                         "of a face box; counted by the oracle (tests/golden/necessary_pairs.py)"}
    for name, make in workloads().items():
        out[name] = count(make())
        print(name, out[name])
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
