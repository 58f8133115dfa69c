"""Writes precision_stress.npz: the grazing displacement of the precision-stress
workload and its grazing fraction, both from the oracle.

The workload: 128^3 order-3 hexes (64 nodes each, h = 1/32) on [-2,2]^3 cut by
a sphere of radius 1 made of 6*32*32 order-3 faces, with some lattice vertices
near the sphere moved so close to the surface that FP32 arithmetic alone
cannot tell how far they are (Sec. 4.2: only the prepass is said to tolerate
single precision).  A vertex within 2h of the unit sphere is picked with
probability pi_g (one seeded uniform per vertex, so a larger pi_g picks a
superset); a picked vertex is moved along its ray from the centre onto the
linearised surface (the ray's hit on the triangles of the four faces nearest
in direction) and then off it by delta ~ U(-1e-4 h, 1e-4 h) along the hit
triangle's normal.

The necessary pair set S* (tests/golden/necessary_pairs.py) is the set of
element-face pairs any box-pruned exact method must evaluate: over the
elements whose node box lies within tol of a face node box,
S*(E) = {F : boxdist(E, F) <= d(E)}.  A pair is grazing when its distance
d(E, F) (oracle.pair_dist) is positive and below 1e-4 h -- near contact
without crossing, where FP32 cannot settle the pair.  pi_g is found by a fixed
bisection (8 steps on [0, 0.2]) so that about 5 % of the S* pairs are grazing.

Stored: pi_g, the moved vertex indices (into the flat (385^3) lattice) and
their coordinates, the signed offsets delta, the oracle's point-surface
distance of a sample of moved vertices (a check of the construction), the S*
size, the grazing and crossing counts, and digests of the faces.

Calls only the oracle and the seeded input generators.  Run from the
repository root (about ten minutes on eight cores):
    python tests/golden/precision_stress.py
"""
from __future__ import annotations

import hashlib
import importlib.util
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "precision_stress.npz")
N, P, M, Q = 128, 3, 32, 3
TOL = 1e-7
SEED = 44
TARGET = 0.05


def sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _np():
    spec = importlib.util.spec_from_file_location("necessary_pairs", os.path.join(HERE, "necessary_pairs.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


class Setup:
    """The unmoved lattice, the surface and the per-vertex draws."""

    def __init__(self):
        sys.path.insert(0, ROOT)
        import oracle as O
        import workloads as W
        self.O, self.W = O, W
        self.h = 4.0 / N
        self.faces = W.cubed_sphere(M, Q, radius=1.0)
        self.lat = W.hex_lattice(N, P)
        flat = self.lat.reshape(-1, 3)
        r = np.sqrt((flat * flat).sum(axis=1))
        self.cand = np.nonzero(np.abs(r - 1.0) < 2.0 * self.h)[0]
        g = np.random.default_rng(SEED)
        self.u = g.random(self.cand.size)
        self.delta = g.uniform(-1e-4 * self.h, 1e-4 * self.h, size=self.cand.size)
        self.tris = O.surface_tris(Q, self.faces)               # [F * 2q^2][3][3]
        fc = self.faces.reshape(self.faces.shape[0], -1, 3).mean(axis=1)
        self.fdir = fc / np.sqrt((fc * fc).sum(axis=1, keepdims=True))

    def moved(self, pi_g):
        """(indices into the flat lattice, new coordinates, delta) for pi_g."""
        sel = np.nonzero(self.u < pi_g)[0]
        idx = self.cand[sel]
        flat = self.lat.reshape(-1, 3)
        per = 2 * Q * Q
        new = np.empty((idx.size, 3))
        ok_all = np.zeros(idx.size, dtype=bool)
        for s in range(0, idx.size, 4096):
            x = flat[idx[s:s + 4096]]
            dd = x / np.sqrt((x * x).sum(axis=1, keepdims=True))
            near = np.argpartition(-(dd @ self.fdir.T), 4, axis=1)[:, :4]
            T = self.tris[(near[:, :, None] * per + np.arange(per)).reshape(dd.shape[0], -1)]
            a, b, c = T[:, :, 0], T[:, :, 1], T[:, :, 2]
            e1, e2 = b - a, c - a
            pv = np.cross(dd[:, None, :], e2)
            det = (e1 * pv).sum(-1)
            inv = 1.0 / np.where(np.abs(det) > 1e-300, det, 1e-300)
            tv = -a
            u = (tv * pv).sum(-1) * inv
            qv = np.cross(tv, e1)
            v = (dd[:, None, :] * qv).sum(-1) * inv
            t = (e2 * qv).sum(-1) * inv
            hit = (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0) & (np.abs(det) > 1e-300)
            t = np.where(hit, t, np.inf)
            k = np.argmin(t, axis=1)
            rows = np.arange(dd.shape[0])
            tk = t[rows, k]
            nrm = np.cross(e1[rows, k], e2[rows, k])
            nrm /= np.sqrt((nrm * nrm).sum(-1, keepdims=True))
            cosang = (nrm * dd).sum(-1)
            dl = self.delta[sel[s:s + 4096]]
            tt = tk + dl / np.where(np.abs(cosang) > 0.5, cosang, 1.0)
            new[s:s + 4096] = dd * tt[:, None]
            ok_all[s:s + 4096] = np.isfinite(tk)
        return idx[ok_all], new[ok_all], self.delta[sel][ok_all]

    def nodes(self, idx, new):
        lat = self.lat.copy()
        lat.reshape(-1, 3)[idx] = new
        return self.W.gather_elements(lat, N, P)

    def grazing(self, nodes):
        """(|S*|, grazing pairs, crossing pairs, exact-test elements)."""
        O = self.O
        NP = _np()
        ids = NP.exact_test_elements(nodes, self.faces)
        _, dist, _, st = O.cut(P, nodes, Q, self.faces, ids=ids, tol=TOL)
        assert st["undecidable"] == 0
        d = np.abs(dist)
        eb = np.concatenate([nodes[ids].min(1), nodes[ids].max(1)], 1)
        fb = np.concatenate([self.faces.min(1), self.faces.max(1)], 1)
        E, F = [], []
        for s in range(0, ids.size, 2048):
            a = eb[s:s + 2048]
            gap = np.maximum(0.0, np.maximum(a[:, None, :3] - fb[None, :, 3:], fb[None, :, :3] - a[:, None, 3:]))
            bd = np.sqrt((gap * gap).sum(-1))
            e, f = np.nonzero(bd <= d[s:s + 2048, None])
            E.append(ids[s + e])
            F.append(f)
        E, F = np.concatenate(E), np.concatenate(F)
        pd = O.pair_dist(P, nodes, Q, self.faces, E, F)
        graze = int(((pd > 0) & (pd < 1e-4 * self.h)).sum())
        cross = int((pd == 0).sum())
        return int(E.size), graze, cross, int(ids.size)


def main():
    t0 = time.time()
    S = Setup()
    print(f"{S.cand.size} lattice vertices within 2h of the sphere ({time.time() - t0:.0f} s)")
    lo, hi = 0.0, 0.2
    best = None
    for it in range(8):
        mid = 0.5 * (lo + hi)
        idx, new, dl = S.moved(mid)
        nodes = S.nodes(idx, new)
        n_s, graze, cross, n_ex = S.grazing(nodes)
        frac = graze / n_s
        print(f"pi_g {mid:.5f}: {idx.size} moved, |S*| {n_s}, grazing {graze} ({100 * frac:.2f} %), "
              f"crossing {cross}, exact-test elements {n_ex} ({time.time() - t0:.0f} s)")
        if best is None or abs(frac - TARGET) < abs(best[1] - TARGET):
            best = (mid, frac, idx, new, dl, n_s, graze, cross, n_ex)
        if frac < TARGET:
            lo = mid
        else:
            hi = mid
    mid, frac, idx, new, dl, n_s, graze, cross, n_ex = best
    # the construction, checked by the oracle's point-surface distance on a
    # sample of moved vertices: |distance| within rounding of |delta|
    g = np.random.default_rng(1)
    smp = g.choice(idx.size, size=min(200, idx.size), replace=False)
    chk = np.array([S.O.point_surface(new[k], S.tris)[0] for k in smp])
    err = np.abs(chk - np.abs(dl[smp]))
    print(f"chosen pi_g {mid:.5f}: grazing {100 * frac:.2f} %; point-surface check max |d - |delta|| "
          f"{err.max():.3e} (h = {S.h})")
    np.savez_compressed(OUT, pi_g=np.array(mid), idx=idx.astype(np.int64), coords=new, delta=dl,
                        check_ids=smp.astype(np.int64), check_dist=chk, s_star_pairs=np.array(n_s),
                        grazing_pairs=np.array(graze), crossing_pairs=np.array(cross),
                        exact_test_elements=np.array(n_ex), faces_sha256=np.array(sha(S.faces)),
                        n=np.array(N), p=np.array(P), m=np.array(M), q=np.array(Q))
    print(f"wrote {OUT} ({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    main()
