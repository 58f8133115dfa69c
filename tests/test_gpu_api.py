"""C-ABI behaviour on the GPU: batched cuts equal single cuts, serving tickets,
host vs device buffers, errors surfacing as status codes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
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


def test_host_buffers_equal_device_buffers():
    c = W.sphere_in_box(n=12, p=2, m=6, q=2, seed=21)
    with dc.Context([(c.p, c.nodes)]) as ctx:
        fh = np.empty(c.n_elem, dtype=np.int8)
        dh = np.empty(c.n_elem)
        ctx.cut(0, c.q, c.faces, fh, dh)
        dev = torch.device("cuda:0")
        fd = torch.empty(c.n_elem, dtype=torch.int8, device=dev)
        dd = torch.empty(c.n_elem, dtype=torch.float64, device=dev)
        ctx.cut(0, c.q, torch.from_numpy(c.faces).to(dev), fd, dd)
        torch.cuda.synchronize()
    assert np.array_equal(fh, fd.cpu().numpy()) and np.array_equal(dh, dd.cpu().numpy())
    rf, _, _, _ = O.cut(c.p, c.nodes, c.q, c.faces)
    assert np.array_equal(fh, rf)


def test_batch_equals_single_cuts():
    cases = W.batch_cases(count=7, seed=5, n_range=(5, 14), m_choices=(4, 6, 8))
    meshes = [(cs.p, cs.nodes) for cs in cases]
    with dc.Context(meshes) as ctx:
        singles = []
        for i, cs in enumerate(cases):
            f = np.empty(cs.n_elem, dtype=np.int8)
            d = np.empty(cs.n_elem)
            ctx.cut(i, cs.q, cs.faces, f, d, pose=cs.pose)
            singles.append((f, d))
        outs = [(np.empty(cs.n_elem, dtype=np.int8), np.empty(cs.n_elem)) for cs in cases]
        reqs = [dict(q=cs.q, faces=cs.faces, flags_out=o[0], dist_out=o[1], pose=cs.pose) for cs, o in zip(cases, outs)]
        ctx.cut_batch(list(range(len(cases))), reqs)
        st = ctx.stats()
    for (f1, d1), (f2, d2) in zip(singles, outs):
        assert np.array_equal(f1, f2) and np.array_equal(d1, d2)
    assert st["n_elem"] == sum(cs.n_elem for cs in cases)
    # and the batch matches the oracle on two of its instances
    for i in (0, 3):
        cs = cases[i]
        rf, _, _, _ = O.cut(cs.p, cs.nodes, cs.q, cs.faces, pose=cs.pose)
        assert np.array_equal(outs[i][0], rf)


def test_submit_poll_overlap_matches_cut():
    cases = [W.sphere_in_box(n=n, p=2, m=m, q=2, seed=30 + n) for n, m in ((10, 6), (14, 8), (8, 4))]
    with dc.Context([(cs.p, cs.nodes) for cs in cases], max_inflight=4) as ctx:
        ref = [ctx.cut(i, cs.q, cs.faces) for i, cs in enumerate(cases)]
        outs = [np.full(cs.n_elem, 9, dtype=np.int8) for cs in cases]
        tickets = [ctx.submit(i, cs.q, cs.faces, outs[i]) for i, cs in enumerate(cases)]
        with pytest.raises(dc.DirectCutError) as ei:
            ctx.submit(0, cases[0].q, cases[0].faces, np.empty(cases[0].n_elem, dtype=np.int8))
        assert ei.value.status == dc.DC_EBUSY
        for t in tickets:
            assert ctx.poll(t, timeout_us=-1) == 0
        with pytest.raises(dc.DirectCutError) as ei:
            ctx.poll(tickets[0], 0)
        assert ei.value.status == dc.DC_ENOTFOUND
    for a, b in zip(ref, outs):
        assert np.array_equal(a, b)


def test_invalid_arguments_are_status_codes():
    c = W.sphere_in_box(n=4, p=1, m=2, q=1, seed=2)
    with dc.Context([(c.p, c.nodes)]) as ctx:
        bad = c.faces.copy()
        bad[0, 0, 0] = np.nan
        for kw, st in ((dict(q=5), dc.DC_EINVAL), (dict(faces=bad), dc.DC_EINVAL), (dict(mesh=3), dc.DC_ENOTFOUND)):
            args = dict(mesh=0, q=c.q, faces=c.faces)
            args.update(kw)
            with pytest.raises(dc.DirectCutError) as ei:
                ctx.cut(args["mesh"], args["q"], args["faces"])
            assert ei.value.status == st
        # the context stays usable after errors
        f = ctx.cut(0, c.q, c.faces)
        rf, _, _, _ = O.cut(c.p, c.nodes, c.q, c.faces)
        assert np.array_equal(f, rf)
    with pytest.raises(dc.DirectCutError) as ei:
        dc.Context([(5, c.nodes)])
    assert ei.value.status == dc.DC_EINVAL
    nodes = c.nodes.copy()
    nodes[1, 2, 1] = np.inf
    with pytest.raises(dc.DirectCutError) as ei:
        dc.Context([(1, nodes)])
    assert ei.value.status == dc.DC_EINVAL


@pytest.mark.parametrize("value", [np.nan, -np.nan, np.inf, -np.inf, 1e301, -1e301, 1e300])
def test_huge_or_non_finite_coordinates_are_rejected(value):
    # the grid's node boxes and the surface's face boxes are reduced on
    # integer keys of the bit patterns; a coordinate of magnitude 1e300 or
    # more, or not finite, anywhere in an element or a face, is an error
    c = W.sphere_in_box(n=5, p=2, m=2, q=2, seed=4)
    npe = c.nodes.shape[1]
    for e, nd, a in ((0, 0, 0), (c.n_elem - 1, npe - 1, 2), (57, 13, 1)):
        nodes = c.nodes.copy()
        nodes[e, nd, a] = value
        with pytest.raises(dc.DirectCutError) as ei:
            dc.Context([(c.p, nodes)])
        assert ei.value.status == dc.DC_EINVAL, (e, nd, a)
    with dc.Context([(c.p, c.nodes)]) as ctx:
        npf = c.faces.shape[1]
        for f, nd, a in ((0, 0, 0), (c.n_faces - 1, npf - 1, 2), (5, 4, 1)):
            faces = c.faces.copy()
            faces[f, nd, a] = value
            with pytest.raises(dc.DirectCutError) as ei:
                ctx.cut(0, c.q, faces)
            assert ei.value.status == dc.DC_EINVAL, (f, nd, a)
        # and the context still cuts
        f = ctx.cut(0, c.q, c.faces)
        rf, _, _, _ = O.cut(c.p, c.nodes, c.q, c.faces)
        assert np.array_equal(f, rf)


def test_memory_budget_admission():
    c = W.sphere_in_box(n=8, p=2, m=4, q=2, seed=3)
    # nodes, float boxes, float element-frame nodes, frame origins
    mesh_bytes = c.nodes.nbytes + c.n_elem * 24 + c.nodes.nbytes // 2 + c.n_elem * 24
    with pytest.raises(dc.DirectCutError) as ei:
        dc.Context([(c.p, c.nodes)], mem_budget_bytes=mesh_bytes // 2)
    assert ei.value.status == dc.DC_ENOMEM
    with dc.Context([(c.p, c.nodes)], mem_budget_bytes=mesh_bytes + 1024) as ctx:
        with pytest.raises(dc.DirectCutError) as ei:
            ctx.cut(0, c.q, c.faces)
        assert ei.value.status == dc.DC_EBUSY


def test_graph_replay_equals_direct_launches(monkeypatch):
    """Cuts replayed from captured CUDA graphs equal directly launched cuts,
    across repeated requests of one shape and a change of shape."""
    cases = [W.sphere_in_box(n=10, p=2, m=6, q=2, seed=41), W.sphere_in_box(n=10, p=2, m=4, q=2, seed=42)]
    outs = {}
    for mode in ("graphs", "direct"):
        if mode == "direct":
            monkeypatch.setenv("DC_NO_GRAPHS", "1")
        with dc.Context([(cases[0].p, cases[0].nodes)]) as ctx:
            res = []
            for cs in (cases[0], cases[1], cases[0], cases[0]):
                f = np.empty(cs.n_elem, dtype=np.int8)
                d = np.empty(cs.n_elem)
                ctx.cut(0, cs.q, cs.faces, f, d)
                res.append((f, d))
            outs[mode] = res
    for (f1, d1), (f2, d2) in zip(outs["graphs"], outs["direct"]):
        assert np.array_equal(f1, f2) and np.array_equal(d1, d2)
    assert np.array_equal(outs["graphs"][0][0], outs["graphs"][2][0])


def test_stats_count_the_flags():
    """n_fringe + n_hole + n_field cover every element and equal the flag
    counts, with and without distances (the flags-only split and the full
    search)."""
    c = W.sphere_in_box(n=14, p=2, m=6, q=2, seed=23)
    with dc.Context([(c.p, c.nodes)]) as ctx:
        for want_dist in (False, True):
            f = np.empty(c.n_elem, dtype=np.int8)
            d = np.empty(c.n_elem) if want_dist else None
            ctx.cut(0, c.q, c.faces, f, d)
            st = ctx.stats()
            assert st["n_elem"] == c.n_elem
            assert st["n_fringe"] == int((f == dc.DC_FRINGE).sum())
            assert st["n_hole"] == int((f == dc.DC_HOLE).sum())
            assert st["n_field"] == int((f == dc.DC_FIELD).sum())
            assert 0 <= st["n_full_search"] <= st["n_candidates"]
            if want_dist:
                assert st["near_tasks"] == 0 and st["n_full_search"] == st["n_candidates"]
