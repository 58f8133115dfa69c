"""The batching and serving workloads at their stated sizes, checked element by
element: every element of every instance and of every request takes the flag
the FP64 CPU oracle gives it (elements far from the surface by the closed form
of tests/sphere_split.py, every other element by the oracle itself).

Batching: 256 independent instances (8^3 to 40^3 Q2 hexes, cubed spheres of
6*m*m Q2 faces with m in {8, 16, 24, 32}, random rotation and offset each) in
one batched cut.  Serving: resident 32^3, 64^3 and 96^3 Q2 grids, a seeded
stream of requests from a dimpled sphere turning 0.5 degrees per step,
admitted through dc_submit / dc_poll with several requests in flight.
"""
import os
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import sphere_split as SS
import workloads as W

pytestmark = pytest.mark.gpu
dc = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global dc
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1711_07663_gb300 as m
    from paper_1711_07663_gb300 import build as B
    B.build()
    m.load()
    dc = m


def separated(flags, n):
    """Fringe separates hole from field: no hole element touches a field element."""
    G = flags.reshape(n, n, n)
    for ax in range(3):
        a = np.moveaxis(G, ax, 0)
        lo, hi = a[:-1], a[1:]
        if np.any((lo == O.HOLE) & (hi == O.FIELD)) or np.any((lo == O.FIELD) & (hi == O.HOLE)):
            return False
    return True


def test_batch_256_instances_in_one_cut():
    cases = W.batch_cases()
    assert len(cases) == 256
    meshes = [(cs.p, cs.nodes) for cs in cases]
    outs = [np.full(cs.n_elem, 9, dtype=np.int8) for cs in cases]
    with dc.Context(meshes) as ctx:
        reqs = [dict(q=cs.q, faces=cs.faces, flags_out=o, pose=cs.pose) for cs, o in zip(cases, outs)]
        ctx.cut_batch(list(range(len(cases))), reqs)
        st = ctx.stats()
        # a second batched cut of the same requests gives the same flags
        again = [np.full(cs.n_elem, 9, dtype=np.int8) for cs in cases]
        ctx.cut_batch(list(range(len(cases))), [dict(r, flags_out=a) for r, a in zip(reqs, again)])
    assert st["n_elem"] == sum(cs.n_elem for cs in cases)
    assert st["n_fringe"] + st["n_hole"] + st["n_field"] == st["n_elem"]
    checked = 0
    for i, (cs, f) in enumerate(zip(cases, outs)):
        assert np.array_equal(f, again[i])
        assert separated(f, cs.n), cs.name
        # every element of every instance: the sphere (radius 1 about the
        # origin before the pose) by closed form away from it, the oracle near it
        ref, k = SS.expected_flags(O, cs.p, cs.nodes, cs.q, cs.faces, cs.centre, pose=cs.pose)
        checked += k
        bad = np.nonzero(f != ref)[0]
        assert bad.size == 0, f"{cs.name}: elements {bad[:10]} gpu {f[bad[:10]]} expected {ref[bad[:10]]}"
    print(f"batch: {st['n_elem']} elements of 256 instances equal, {checked} of them by the oracle")


def test_serving_stream_of_turning_sphere():
    meshes = [W.background(n, 2, sinusoid=0.1) for n in (32, 64, 96)]
    sizes = (32, 64, 96)
    base = W.dimpled_sphere_case(n=8, m=32, q=2)  # its surface: the dimpled sphere of 6144 Q2 faces
    faces = base.faces
    centre = base.centre
    g = np.random.default_rng(77)
    axis = g.normal(size=3)
    n_req = 32
    which = g.choice(3, size=n_req, p=[0.5, 0.3, 0.2])
    poses = []
    for k in range(n_req):
        R = W.axis_rotation(axis, np.deg2rad(0.5 * k))
        poses.append(np.concatenate([R, np.zeros((3, 1))], axis=1))
    with dc.Context([(2, m) for m in meshes], max_inflight=4) as ctx:
        outs = [np.full(meshes[w].shape[0], 9, dtype=np.int8) for w in which]
        lat = []
        pending = {}
        k = 0
        t0 = time.perf_counter()
        while k < n_req or pending:
            # admit while a slot is free, then collect whatever has finished
            while k < n_req:
                try:
                    tk = ctx.submit(int(which[k]), 2, faces, outs[k], pose=poses[k])
                except dc.DirectCutError as e:
                    assert e.status == dc.DC_EBUSY
                    break
                pending[tk] = (k, time.perf_counter())
                k += 1
            for tk in list(pending):
                rc = ctx.poll(tk, timeout_us=0 if k < n_req else -1)
                if rc == 0:
                    lat.append(time.perf_counter() - pending.pop(tk)[1])
        wall = time.perf_counter() - t0
        # every request equals the synchronous cut of the same pose
        for k in range(n_req):
            ref = ctx.cut(int(which[k]), 2, faces, pose=poses[k])
            assert np.array_equal(ref, outs[k]), f"request {k}"
    lat = np.array(lat) * 1e3
    print(f"serving: {n_req} requests, p50 {np.percentile(lat, 50):.3f} ms, p99 {np.percentile(lat, 99):.3f} ms, "
          f"{n_req / wall:.1f} req/s (host polling loop)")
    # every element of every request against the oracle (closed form far
    # from the surface)
    checked = 0
    for k in range(n_req):
        w = int(which[k])
        ref, nk = SS.expected_flags(O, 2, meshes[w], 2, faces, centre, pose=poses[k])
        checked += nk
        bad = np.nonzero(outs[k] != ref)[0]
        assert bad.size == 0, f"request {k}: elements {bad[:10]}"
        assert separated(outs[k], sizes[w])
    print(f"serving: every element of {n_req} requests equals the oracle ({checked} by the oracle itself)")


def test_submit_copies_pinned_host_faces_before_returning():
    """dc_submit owns its inputs once it returns: a pinned host face buffer
    overwritten right after the call must not change the submitted cut."""
    case = W.dimpled_sphere_case(n=32, m=16, seed=12)
    nodes = torch.from_numpy(case.nodes).cuda()
    faces_pinned = torch.from_numpy(case.faces.copy()).pin_memory()
    pose = np.concatenate([W.axis_rotation([0.3, 0.2, 0.9], 0.2), np.array([[0.02], [0.0], [-0.03]])], axis=1)
    with dc.Context([(case.p, nodes)], max_inflight=3) as ctx:
        ref = ctx.cut(0, case.q, case.faces, pose=pose)
        outs = [torch.full((case.n_elem,), 9, dtype=torch.int8).pin_memory() for _ in range(2)]
        tickets = []
        for o in outs:
            faces_pinned.copy_(torch.from_numpy(case.faces))
            tickets.append(ctx.submit(0, case.q, faces_pinned, o, pose=pose))
            faces_pinned.mul_(0.5)   # the caller reuses its buffer at once
        for t in tickets:
            assert ctx.poll(t, timeout_us=-1) == 0
    for o in outs:
        assert np.array_equal(o.numpy(), ref)
    ids = np.unique(np.concatenate([np.nonzero(ref == O.FRINGE)[0][:200],
                                    np.random.default_rng(3).choice(case.n_elem, 100, replace=False)]))
    rf, _, _, rst = O.cut(case.p, case.nodes, case.q, case.faces, pose=pose, ids=ids)
    assert rst["undecidable"] == 0
    assert np.array_equal(ref[ids], rf)


def precision_stress_case():
    """The 128^3 Q3 grid with the grazing vertices the oracle-side script
    placed (tests/golden/precision_stress.npz) and the Q3 sphere of 6*32*32
    faces; returns (nodes, faces, moved-vertex mask of the elements, stored)."""
    G = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "precision_stress.npz"))
    n, p, m, q = int(G["n"]), int(G["p"]), int(G["m"]), int(G["q"])
    lat = W.hex_lattice(n, p)
    lat.reshape(-1, 3)[G["idx"]] = G["coords"]
    gi = W.gather_index(n, p)
    nodes = np.ascontiguousarray(lat.reshape(-1, 3)[gi])
    moved = np.zeros(lat.shape[0] * lat.shape[1] * lat.shape[2], dtype=bool)
    moved[G["idx"]] = True
    graze = np.nonzero(moved[gi].any(axis=1))[0]
    faces = W.cubed_sphere(m, q, radius=1.0)
    return nodes, faces, graze, G


@pytest.mark.slow
def test_precision_stress_128cube_q3_grazing():
    """FP32 bulk + FP64 re-solve against all-FP64 on the precision-stress
    workload (5 % of the necessary element-face pairs within 1e-4 h of contact
    without crossing): identical flags in both forms, distances within 1e-12
    relative, the FP32 stage's own distances within its rounding bound of the
    FP64 ones, and the oracle on the grazing elements."""
    nodes, faces, graze, G = precision_stress_case()
    n, p, q = int(G["n"]), int(G["p"]), int(G["q"])
    h = 4.0 / n
    dev = torch.device("cuda:0")
    tn = torch.from_numpy(nodes).to(dev)
    tf = torch.from_numpy(faces).to(dev)
    res = {}
    for prec in (dc.DC_FP32_RECHECK, dc.DC_FP64):
        with dc.Context([(p, tn)], precision=prec) as ctx:
            f = torch.empty(nodes.shape[0], dtype=torch.int8, device=dev)
            d = torch.empty(nodes.shape[0], dtype=torch.float64, device=dev)
            d32 = torch.full((nodes.shape[0],), 7.0, dtype=torch.float32, device=dev) \
                if prec == dc.DC_FP32_RECHECK else None
            ctx.cut(0, q, tf, f, d, fp32_dist_out=d32)
            st = ctx.stats()
            f2 = torch.empty_like(f)
            ctx.cut(0, q, tf, f2)  # flags only
            torch.cuda.synchronize()
            res[prec] = (f.cpu().numpy(), d.cpu().numpy(), f2.cpu().numpy(), st,
                         None if d32 is None else d32.cpu().numpy())
    f32, d32, g32, s32, e32 = res[dc.DC_FP32_RECHECK]
    f64, d64, g64, _, _ = res[dc.DC_FP64]
    assert np.array_equal(f32, f64) and np.array_equal(g32, g64) and np.array_equal(f32, g32)
    fin = np.isfinite(d64)
    assert np.array_equal(fin, np.isfinite(d32))
    assert np.all(np.abs(d32[fin] - d64[fin]) <= 1e-12 * np.maximum(np.abs(d64[fin]), h))
    # the FP32 stage's distances: written for every exact-test element (NaN
    # only where none was computed), +-inf where the hole map decided, and
    # within the FP32 rounding bound (64 u S, S below 2 h here) of FP64
    assert not np.any(e32 == 7.0)
    assert np.array_equal(np.isinf(e32), ~fin)
    have = fin & ~np.isnan(e32)
    assert have.sum() > 1000
    err = np.abs(e32[have].astype(np.float64) - d64[have])
    assert np.all(err <= 64 * 2.0 ** -24 * 2 * h), f"max FP32 error {err.max() / h:.3e} h"
    grazing = np.abs(d64[fin]) < 1e-4 * h
    print(f"precision stress: {nodes.shape[0]} elements, {s32['n_candidates']} candidates, "
          f"{int(grazing.sum())} elements with |d| < 1e-4 h, grazing pairs {int(G['grazing_pairs'])} of "
          f"{int(G['s_star_pairs'])} S* pairs, {s32['pairs_recheck']} FP64 re-solves of {s32['pairs_bulk']} FP32 "
          f"pairs, max |d32 - d64| {err.max() / h:.3e} h; flags FP32+re-check == FP64")
    g = np.random.default_rng(44)
    ids = np.unique(np.concatenate([g.choice(graze, size=min(240, graze.size), replace=False),
                                    g.choice(np.nonzero(fin)[0], size=60, replace=False)]))
    rf, rd, _, rst = O.cut(p, nodes, q, faces, ids=ids)
    assert rst["undecidable"] == 0
    assert np.array_equal(f32[ids], rf)
    ok = np.isfinite(d32[ids])
    assert np.all(np.abs(d32[ids][ok] - rd[ok]) <= 1e-12 * np.maximum(np.abs(rd[ok]), h))
