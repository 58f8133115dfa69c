"""Pins of the set logic after the cut (oracle/overset.py): removal per cut
kind, union, artificial-boundary faces and the unblank procedure, against the
paper's sentences restated case by case, brute-force lattice counts and the
invariants of a sphere moving through a grid."""
import itertools

import numpy as np

import oracle as O
from oracle import overset as S
import workloads as W

STATES = (S.HOLE, S.FIELD, S.FRINGE)


def test_removed_per_cut_kind():
    f = np.array([S.HOLE, S.FIELD, S.FRINGE], dtype=np.int8)
    # a wall removes what lies inside it and what it passes through
    assert S.removed(f, S.WALL).tolist() == [True, False, True]
    # an overset boundary removes only what lies inside it
    assert S.removed(f, S.OVERSET).tolist() == [True, False, False]


def test_union_removes_what_any_cut_removes():
    a = np.array([S.HOLE, S.FIELD, S.FIELD, S.FRINGE, S.FRINGE], dtype=np.int8)
    b = np.array([S.FIELD, S.FIELD, S.HOLE, S.FIELD, S.FRINGE], dtype=np.int8)
    assert S.union([a, b], [S.OVERSET, S.OVERSET]).tolist() == [True, False, True, False, False]
    assert S.union([a, b], [S.WALL, S.OVERSET]).tolist() == [True, False, True, True, True]
    assert S.union([a], [S.WALL]).tolist() == S.removed(a, S.WALL).tolist()


def test_unblank_follows_the_algorithm_sentence_by_sentence():
    for kind in (S.WALL, S.OVERSET):
        for ft, ftp, prev in itertools.product(STATES, STATES, (False, True)):
            now, unb = S.unblank(np.array([prev]), np.array([ft], np.int8), np.array([ftp], np.int8), kind)
            hole_t, hole_tp = bool(S.removed([ft], kind)[0]), bool(S.removed([ftp], kind)[0])
            if kind == S.WALL:
                # "any cell which becomes a hole cell in I_t+ can be set to hole in I_t"
                want_now = hole_t or hole_tp
                # "any hole cell in I_t- which is no longer a hole cell in I_t and I_t+ must be unblanked"
                want_unb = prev and (not hole_t) and (not hole_tp)
            else:
                # cells are not blanked until both cuts agree they are no longer needed
                want_now = hole_t and hole_tp
                # "any hole cell in I_t- which is no longer a hole cell in I_t or I_t+ must be unblanked"
                want_unb = prev and ((not hole_t) or (not hole_tp))
            assert bool(now[0]) == want_now, (kind, ft, ftp, prev)
            assert bool(unb[0]) == want_unb, (kind, ft, ftp, prev)


def test_structured_neighbours_are_symmetric():
    nb = S.structured_neighbours(3, 4, 5)
    n = 3 * 4 * 5
    for e in range(n):
        for j in range(6):
            o = nb[e, j]
            if o >= 0:
                assert nb[o, j ^ 1] == e
    # boundary faces: 2 (ny nz + nx nz + nx ny)
    assert int((nb < 0).sum()) == 2 * (4 * 5 + 3 * 5 + 3 * 4)


def test_ab_faces_against_lattice_pair_counts():
    g = np.random.default_rng(3)
    nx, ny, nz = 5, 4, 6
    nb = S.structured_neighbours(nx, ny, nz)
    # one removed element: its 6 neighbours each carry the face pointing at it
    rem = np.zeros(nx * ny * nz, dtype=bool)
    c = 2 + nx * (1 + ny * 2)
    rem[c] = True
    mask = S.ab_faces(rem, nb)
    assert int(sum(bin(int(m)).count("1") for m in mask)) == 6
    for j in range(6):
        assert mask[nb[c, j]] == np.uint8(1 << (j ^ 1))
    # random removal: the number of AB faces is the number of kept-removed
    # face pairs of the lattice
    for _ in range(5):
        rem = g.random(nx * ny * nz) < 0.3
        mask = S.ab_faces(rem, nb)
        G = rem.reshape(nz, ny, nx)
        pairs = 0
        for ax in range(3):
            a = np.moveaxis(G, 2 - ax, 0)
            pairs += int(np.sum(a[:-1] != a[1:]))
        assert int(sum(bin(int(m)).count("1") for m in mask)) == pairs
        assert np.all(mask[rem] == 0)


def test_moving_sphere_invariants():
    """A sphere moving 0.6 h per step through a 10^3 Q1 grid: wall removal
    covers both cut positions, overset removal neither exceeds them, and the
    unblanked elements are exactly those that leave the removed set (some do,
    over the steps)."""
    n, p, q = 10, 1, 2
    nodes = W.background(n, p, jitter=0.05, seed=5)
    faces = W.cubed_sphere(6, q, radius=1.0)
    h = 4.0 / n
    prev = {S.WALL: np.zeros(n ** 3, bool), S.OVERSET: np.zeros(n ** 3, bool)}
    total = {S.WALL: 0, S.OVERSET: 0}
    for step in range(4):
        pose = lambda k: np.concatenate([np.eye(3), np.array([[0.6 * h * k], [0.0], [0.0]])], axis=1)
        ft, _, _, _ = O.cut(p, nodes, q, faces, pose=pose(step))
        ftp, _, _, _ = O.cut(p, nodes, q, faces, pose=pose(step + 1))
        for kind in (S.WALL, S.OVERSET):
            now, unb = S.unblank(prev[kind], ft, ftp, kind)
            rt, rtp = S.removed(ft, kind), S.removed(ftp, kind)
            if kind == S.WALL:
                assert np.all(now >= rt) and np.all(now >= rtp)
            else:
                assert np.all(now <= rt) and np.all(now <= rtp)
            assert np.array_equal(unb, prev[kind] & ~now)
            total[kind] += int(unb.sum())
            prev[kind] = now
    assert total[S.WALL] > 0 and total[S.OVERSET] > 0
