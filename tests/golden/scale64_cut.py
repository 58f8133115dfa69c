"""Writes scale64_cut.npz: the oracle's cut of the whole 64^3 scale workload.

The workload is the benchmark's: 262,144 order-2 hexes on [-2,2]^3 curved by
the sinusoidal node displacement, cut by the dimpled sphere of 6144 order-2
faces (workloads.dimpled_sphere_case() with its defaults).  The oracle
classifies every element by the plain definition of the cut (Sec. 4.2:
element-surface distance <= tol is fringe, otherwise the side of the closed
surface decides hole or field) and this file keeps:

  flags       int8  [262144]  HOLE 0, FIELD 1, FRINGE -1, every element
  dist_ids    int32 [k]       elements with |d(E)| <= 3 h (h = 1/16), ascending
  dist        f64   [k]       their signed FP64 distances (+ field, - hole, d fringe)
  nodes_sha256, faces_sha256  digests of the generated inputs, so a change in
                              the generators is caught before flags are compared
  flags_sha256                digest of the flags array
  undecidable, paper_rule_disagree   the oracle's own counts (both must be 0)

The GPU only ever reports exact distances for elements the hole map leaves as
candidates, all of which lie within about one element of the surface; 3 h
covers them with room to spare.

Calls only the oracle and the seeded input generators.  Run from the
repository root (about six minutes on eight cores):
    python tests/golden/scale64_cut.py
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "scale64_cut.npz")
TOL = 1e-7
BAND_H = 3.0


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def case():
    sys.path.insert(0, ROOT)
    import workloads as W
    return W.dimpled_sphere_case()


def main():
    sys.path.insert(0, ROOT)
    import oracle as O
    c = case()
    h = 4.0 / c.n
    t0 = time.time()
    flags, dist, _, st = O.cut(c.p, c.nodes, c.q, c.faces, tol=TOL)
    print(f"oracle cut of {c.n_elem} elements: {time.time() - t0:.1f} s, stats {st}")
    keep = np.nonzero(np.abs(dist) <= BAND_H * h)[0].astype(np.int32)
    np.savez_compressed(
        OUT, flags=flags.astype(np.int8), dist_ids=keep, dist=dist[keep].astype(np.float64),
        nodes_sha256=np.array(sha(c.nodes)), faces_sha256=np.array(sha(c.faces)),
        flags_sha256=np.array(sha(flags.astype(np.int8))), tol=np.array(TOL), band_h=np.array(BAND_H),
        undecidable=np.array(st["undecidable"]), paper_rule_disagree=np.array(st["paper_rule_disagree"]))
    print(f"wrote {OUT}: {keep.size} distances, fringe {int((flags == -1).sum())}, "
          f"hole {int((flags == 0).sum())}, field {int((flags == 1).sum())}")


if __name__ == "__main__":
    main()
