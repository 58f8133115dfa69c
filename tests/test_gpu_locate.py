"""Donor search (point connectivity) on the GPU through the C ABI against the
oracle's brute-force version (oracle/oracle.c, orc_locate): the same donor
wherever the oracle's acceptance is not within rounding of flipping, and the
same reference coordinates (both stop Newton at a residual of 1e-10 h)."""
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


def compare(p, nodes, pts, pose=None):
    with dc.PointLocator(p, nodes) as pl:
        donor, ref = pl.locate(pts, pose=pose)
        st = pl.stats()
    od, orf, om = O.locate(p, nodes, pts, pose=pose)
    # acceptance decisions within rounding of the thresholds may go either way
    robust = (np.abs(om[:, 0]) > 1e-13) & (np.abs(om[:, 1]) > 1e-12)
    assert np.array_equal(donor[robust], od[robust]), np.nonzero(robust & (donor != od))[0][:10]
    both = (donor >= 0) & (donor == od)
    assert np.abs(ref[both] - orf[both]).max(initial=0.0) < 1e-8
    # every donor the GPU reports holds the point (oracle map)
    for k in np.nonzero(donor >= 0)[0][:400]:
        x = pts[k] if pose is None else np.asarray(pose)[:, :3].T @ (pts[k] - np.asarray(pose)[:, 3])
        back, _ = O.iso_map(p, nodes[donor[k]], ref[k])
        h = np.ptp(nodes[donor[k]], axis=0).max()
        assert np.linalg.norm(back - x) <= 1e-10 * h * (1 + 1e-6)
        assert np.abs(ref[k]).max() <= 1 + 1e-8
    return donor, ref, od, st


def test_generated_interior_points():
    nodes = W.sphere_shell(6, 3, 2, 1.0, 1.6)
    g = np.random.default_rng(11)
    E = g.integers(0, nodes.shape[0], size=2000)
    xs = g.uniform(-0.97, 0.97, size=(2000, 3))
    pts = np.array([O.iso_map(2, nodes[e], x)[0] for e, x in zip(E, xs)])
    donor, ref, od, st = compare(2, nodes, pts)
    assert np.array_equal(donor, E)
    assert np.abs(ref - xs).max() < 1e-8
    assert st["n_found"] == 2000 and st["n_points"] == 2000
    n = nodes.shape[0]
    assert st["tree_depth"] == int(np.ceil(np.log2(n + 1)))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_shell_points_with_misses(p):
    nodes = W.sphere_shell(5, 2, p, 1.0, 1.6)
    pts = np.concatenate([W.shell_points(3000, 1.0, 1.6, seed=4), W.shell_points(300, 0.3, 0.95, seed=5),
                          W.shell_points(300, 1.65, 2.5, seed=6)])
    donor, ref, od, st = compare(p, nodes, pts)
    assert np.all(donor[3000:] == -1)
    # straight-sided elements cut the sphere's curvature: some shell points
    # fall outside the grid, the same ones for both
    assert (donor[:3000] >= 0).mean() > 0.9
    assert np.array_equal(donor >= 0, od >= 0)


def test_moving_grid_and_device_tensors():
    nodes = W.sphere_shell(5, 3, 2, 1.0, 1.6)
    pts = W.shell_points(2000, 1.01, 1.59, seed=9)
    R = W.axis_rotation([0.2, 0.9, -0.4], 1.1)
    t = np.array([0.3, -0.2, 0.5])
    pose = np.concatenate([R, t[:, None]], axis=1)
    moved = np.ascontiguousarray(pts @ R.T + t)
    d0, r0, _, _ = compare(2, nodes, pts)
    d1, r1, _, _ = compare(2, nodes, moved, pose=pose)
    assert np.array_equal(d0, d1) and np.abs(r0 - r1).max() < 1e-8
    dev = torch.device("cuda:0")
    with dc.PointLocator(2, torch.from_numpy(nodes).to(dev)) as pl:
        dd, rr = pl.locate(torch.from_numpy(moved).to(dev), pose=pose)
        torch.cuda.synchronize()
        assert np.array_equal(dd.cpu().numpy(), d1) and np.allclose(rr.cpu().numpy(), r1, atol=1e-12)
        e, r = pl.locate(np.zeros((0, 3)))
        assert e.shape == (0,)


def gauss_face_points(p, enodes, face, ng):
    """Gauss-Legendre points (ng x ng) on local face `face` of an element."""
    gx, _ = np.polynomial.legendre.leggauss(ng)
    ax, side = face // 2, (-1.0 if face % 2 == 0 else 1.0)
    out = []
    for v in gx:
        for u in gx:
            xi = np.zeros(3)
            free = [d for d in range(3) if d != ax]
            xi[ax] = side
            xi[free[0]], xi[free[1]] = u, v
            out.append(O.iso_map(p, enodes, xi)[0])
    return out


def test_flux_points_of_artificial_boundary_faces():
    """An overset cut of a 20^3 background by a sphere of radius 1.5 leaves
    artificial-boundary faces; their flux points (3x3 Gauss points on each
    face) find donors in a body-fitted shell grid between radii 1 and 1.6."""
    n, p = 20, 2
    bg = W.background(n, p, jitter=0.05, seed=21)
    over = W.cubed_sphere(12, 2, radius=1.5)
    flags, _, _, _ = O.cut(p, bg, 2, over)
    from oracle import overset as S
    rem = S.removed(flags, S.OVERSET)
    mask = S.ab_faces(rem, S.structured_neighbours(n, n, n))
    pts = []
    for e in np.nonzero(mask)[0]:
        for f in range(6):
            if mask[e] >> f & 1:
                pts += gauss_face_points(p, bg[e], f, 3)
    pts = np.ascontiguousarray(np.array(pts))
    assert len(pts) > 1000
    shell = W.sphere_shell(10, 4, 2, 1.0, 1.6)
    donor, ref, od, st = compare(2, shell, pts)
    assert np.all(donor >= 0)


def test_bench_configuration_sampled():
    """The benchmark's donor search: 2^20 shell points in the 49,152-element Q2
    shell turned by a rigid pose, device tensors; the oracle checks a sample."""
    shell = W.sphere_shell(32, 8, 2, 1.0, 1.6)
    pts = W.shell_points(1 << 20, 1.0, 1.6, seed=17)
    pose = np.concatenate([W.axis_rotation([0.1, 0.7, 0.7], 0.3), np.array([[0.05], [-0.02], [0.01]])], axis=1)
    moved = np.ascontiguousarray(pts @ pose[:, :3].T + pose[:, 3])
    dev = torch.device("cuda:0")
    with dc.PointLocator(2, torch.from_numpy(shell).to(dev)) as pl:
        d, r = pl.locate(torch.from_numpy(moved).to(dev), pose=pose)
        torch.cuda.synchronize()
        st = pl.stats()
    d, r = d.cpu().numpy(), r.cpu().numpy()
    assert st["n_found"] == int((d >= 0).sum())
    g = np.random.default_rng(3)
    k = np.sort(g.choice(pts.shape[0], size=3000, replace=False))
    od, orf, om = O.locate(2, shell, moved[k], pose=pose)
    robust = (np.abs(om[:, 0]) > 1e-13) & (np.abs(om[:, 1]) > 1e-12)
    assert np.array_equal(d[k][robust], od[robust])
    both = (d[k] >= 0) & (d[k] == od)
    assert np.abs(r[k][both] - orf[both]).max() < 1e-8
