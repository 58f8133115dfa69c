"""What follows the cut, on the GPU through the C ABI: the union of a wall and
an overset cut, artificial-boundary faces, and the unblank step of a moving
grid, against the oracle's set logic (oracle/overset.py) on oracle cuts."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from oracle import overset as S
import workloads as W

pytestmark = pytest.mark.gpu
dc = None
DEV = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global dc, DEV
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1711_07663_gb300 as m
    from paper_1711_07663_gb300 import build as B
    B.build()
    m.load()
    dc = m
    DEV = torch.device("cuda:0")


def t8(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int8)).to(DEV)


def test_neighbour_helpers_agree():
    assert np.array_equal(dc.structured_neighbours(4, 3, 5), S.structured_neighbours(4, 3, 5))


def test_union_and_ab_faces_of_a_wall_and_an_overset_cut():
    n, p, q = 24, 2, 2
    nodes = W.background(n, p, jitter=0.05, seed=9)
    wall = W.cubed_sphere(6, q, radius=0.6, centre=(-0.7, 0.1, 0.0))
    over = W.cubed_sphere(8, q, radius=1.1, centre=(0.6, -0.1, 0.05))
    with dc.Context([(p, nodes)]) as ctx:
        fw = ctx.cut(0, q, wall)
        fo = ctx.cut(0, q, over)
    rw, _, _, _ = O.cut(p, nodes, q, wall)
    ro, _, _, _ = O.cut(p, nodes, q, over)
    assert np.array_equal(fw, rw) and np.array_equal(fo, ro)
    ib = torch.empty(n ** 3, dtype=torch.int8, device=DEV)
    dc.dc_blank_union([t8(fw), t8(fo)], [dc.DC_WALL, dc.DC_OVERSET], ib)
    want_removed = S.union([rw, ro], [S.WALL, S.OVERSET])
    got = ib.cpu().numpy()
    assert np.array_equal(got == 0, want_removed) and set(np.unique(got).tolist()) <= {0, 1}
    assert want_removed.sum() > 0 and (~want_removed).sum() > 0
    nb = torch.from_numpy(dc.structured_neighbours(n, n, n)).to(DEV)
    mask = torch.empty(n ** 3, dtype=torch.uint8, device=DEV)
    count = dc.dc_ab_faces(ib, nb, mask)
    want = S.ab_faces(want_removed, S.structured_neighbours(n, n, n))
    assert np.array_equal(mask.cpu().numpy(), want)
    assert count == int(sum(bin(int(m)).count("1") for m in want)) > 0
    # a single cut through the union call is that cut's removal
    dc.dc_blank_union([t8(fw)], [dc.DC_WALL], ib)
    assert np.array_equal(ib.cpu().numpy() == 0, S.removed(rw, S.WALL))


def test_unblank_of_a_moving_sphere():
    n, p, q = 20, 2, 2
    h = 4.0 / n
    nodes = W.background(n, p, jitter=0.05, seed=13)
    faces = W.cubed_sphere(8, q, radius=1.0)
    axis = np.array([0.3, 1.0, -0.2])
    poses = [np.concatenate([W.axis_rotation(axis, 0.02 * k), np.array([[0.45 * h * k], [0.1 * h * k], [0.0]])], axis=1)
             for k in range(6)]
    prev = {k: torch.ones(n ** 3, dtype=torch.int8, device=DEV) for k in (dc.DC_WALL, dc.DC_OVERSET)}
    prev_o = {k: np.zeros(n ** 3, dtype=bool) for k in (S.WALL, S.OVERSET)}
    total = 0
    with dc.Context([(p, nodes)]) as ctx:
        for step in range(5):
            ft = np.empty(n ** 3, dtype=np.int8)
            ftp = np.empty(n ** 3, dtype=np.int8)
            # both cut positions in one batched launch on the same resident grid
            ctx.cut_batch([0, 0], [dict(q=q, faces=faces, flags_out=ft, pose=poses[step]),
                                   dict(q=q, faces=faces, flags_out=ftp, pose=poses[step + 1])])
            rt, _, _, _ = O.cut(p, nodes, q, faces, pose=poses[step])
            rtp, _, _, _ = O.cut(p, nodes, q, faces, pose=poses[step + 1])
            assert np.array_equal(ft, rt) and np.array_equal(ftp, rtp)
            for kind, okind in ((dc.DC_WALL, S.WALL), (dc.DC_OVERSET, S.OVERSET)):
                ib = torch.empty(n ** 3, dtype=torch.int8, device=DEV)
                unb = torch.empty(n ** 3, dtype=torch.uint8, device=DEV)
                cnt = dc.dc_unblank(kind, prev[kind], t8(ft), t8(ftp), ib, unb)
                now, want_unb = S.unblank(prev_o[okind], rt, rtp, okind)
                assert np.array_equal(ib.cpu().numpy() == 0, now)
                assert np.array_equal(unb.cpu().numpy().astype(bool), want_unb)
                assert cnt == int(want_unb.sum())
                total += cnt
                prev[kind] = ib
                prev_o[okind] = now
    assert total > 0


def test_unblank_at_scale_matches_set_logic():
    """The 64^3 workload, the surface turned by 0.5 degrees between the two
    cuts: the GPU step equals the set logic applied to the GPU's own flags."""
    c = W.dimpled_sphere_case()
    poses = [np.concatenate([W.axis_rotation([0.2, 0.9, 0.4], np.deg2rad(0.5 * k)), np.array([[0.01 * k], [0.0], [0.0]])],
                            axis=1) for k in range(3)]
    nodes = torch.from_numpy(c.nodes).to(DEV)
    faces = torch.from_numpy(c.faces).to(DEV)
    fl = [torch.empty(c.n_elem, dtype=torch.int8, device=DEV) for _ in range(3)]
    with dc.Context([(c.p, nodes)]) as ctx:
        for k in range(3):
            ctx.cut(0, c.q, faces, fl[k], pose=poses[k])
    torch.cuda.synchronize()
    f = [x.cpu().numpy() for x in fl]
    for kind, okind in ((dc.DC_WALL, S.WALL), (dc.DC_OVERSET, S.OVERSET)):
        prev_rem = S.removed(f[0], okind)
        ib = torch.empty(c.n_elem, dtype=torch.int8, device=DEV)
        unb = torch.empty(c.n_elem, dtype=torch.uint8, device=DEV)
        cnt = dc.dc_unblank(kind, t8(np.where(prev_rem, 0, 1)), fl[1], fl[2], ib, unb)
        now, want_unb = S.unblank(prev_rem, f[1], f[2], okind)
        assert np.array_equal(ib.cpu().numpy() == 0, now)
        assert np.array_equal(unb.cpu().numpy().astype(bool), want_unb) and cnt == int(want_unb.sum())
