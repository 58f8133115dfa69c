"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Flags must be bit-identical.  Distances: elements that reach the exact test
must agree with the oracle within 1e-12 * max(|d|, h); elements decided by
the hole map report -inf (hole) / +inf (field) and the oracle must agree on
their side.  Sizes span several warps / bins / hole-map runs with ragged
tails; the full 262,144-element benchmark workload is checked on every
element against the oracle's stored cut (tests/golden/scale64_cut.npz, written
by tests/golden/scale64_cut.py, which calls only the oracle).
"""
import hashlib
import os

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


def gpu_cut(p, nodes, q, faces, pose=None, want_dist=True, **cfg):
    dev = torch.device("cuda:0")
    tn = torch.from_numpy(np.ascontiguousarray(nodes)).to(dev)
    tf = torch.from_numpy(np.ascontiguousarray(faces)).to(dev)
    n = nodes.shape[0]
    flags = torch.full((n,), 7, dtype=torch.int8, device=dev)
    dist = torch.full((n,), np.nan, dtype=torch.float64, device=dev) if want_dist else None
    with dc.Context([(p, tn)], **cfg) as ctx:
        ctx.cut(0, q, tf, flags, dist, pose=pose)
        torch.cuda.synchronize()
        st = ctx.stats()
    return flags.cpu().numpy(), (dist.cpu().numpy() if want_dist else None), st


def check(flags, dist, ref_f, ref_d, h):
    bad = np.nonzero(flags != ref_f)[0]
    assert bad.size == 0, f"{bad.size} flag mismatches, first {bad[:8]}: gpu {flags[bad[:8]]} oracle {ref_f[bad[:8]]}"
    if dist is None:
        return
    assert not np.any(np.isnan(dist))
    fin = np.isfinite(dist)
    err = np.abs(dist[fin] - ref_d[fin])
    tol = 1e-12 * np.maximum(np.abs(ref_d[fin]), h)
    assert np.all(err <= tol), f"max dist error {err.max():.3e}"
    # elements settled by the hole map: side agrees, never fringe
    inf = ~fin
    assert np.all(ref_f[inf] != O.FRINGE)
    assert np.all((dist[inf] < 0) == (ref_f[inf] == O.HOLE))


PRECISIONS = [pytest.param(1, id="fp32+recheck"), pytest.param(0, id="fp64")]


@pytest.mark.parametrize("precision", PRECISIONS)
def test_plain_sphere_16cube_q2(precision):
    """The 4096-element plain workload: 16^3 Q2 hexes, jitter 0.05h, cubed
    sphere R=1 of 384 Q2 faces at a seeded offset -- every element."""
    c = W.sphere_in_box(n=16, p=2, m=8, q=2, seed=1)
    f, d, st = gpu_cut(c.p, c.nodes, c.q, c.faces, precision=precision)
    rf, rd, _, rst = O.cut(c.p, c.nodes, c.q, c.faces)
    assert rst["undecidable"] == 0
    check(f, d, rf, rd, 4.0 / c.n)
    assert st["n_candidates"] > 0 and st["n_candidates"] < c.n_elem


@pytest.mark.parametrize("p,q,n,m", [(1, 1, 12, 5), (1, 2, 10, 4), (2, 1, 9, 6), (3, 3, 7, 3), (4, 2, 5, 3),
                                     (2, 4, 6, 2), (3, 1, 6, 7)])
def test_orders(p, q, n, m):
    c = W.sphere_in_box(n=n, p=p, m=m, q=q, seed=10 * p + q, jitter=0.08)
    f, d, _ = gpu_cut(c.p, c.nodes, c.q, c.faces)
    rf, rd, _, rst = O.cut(c.p, c.nodes, c.q, c.faces)
    assert rst["undecidable"] == 0
    check(f, d, rf, rd, 4.0 / n)


def test_dimpled_posed_and_curved():
    c = W.dimpled_sphere_case(n=14, p=2, m=8, q=2, n_dimples=80, seed=4)
    pose = np.concatenate([W.random_rotation(W.rng(9)), np.array([[0.07], [-0.03], [0.05]])], axis=1)
    f, d, _ = gpu_cut(c.p, c.nodes, c.q, c.faces, pose=pose)
    rf, rd, _, _ = O.cut(c.p, c.nodes, c.q, c.faces, pose=pose)
    check(f, d, rf, rd, 4.0 / c.n)


def test_flags_without_distance_output():
    c = W.sphere_in_box(n=12, p=2, m=6, q=2, seed=3)
    f, _, _ = gpu_cut(c.p, c.nodes, c.q, c.faces, want_dist=False)
    rf, _, _, _ = O.cut(c.p, c.nodes, c.q, c.faces)
    check(f, None, rf, None, 4.0 / c.n)


@pytest.mark.parametrize("cells,bins", [(8, 1), (23, 3), (80, 16), (64, 2)])
def test_hole_map_resolution_does_not_change_results(cells, bins):
    c = W.sphere_in_box(n=10, p=2, m=6, q=2, seed=6)
    f, d, _ = gpu_cut(c.p, c.nodes, c.q, c.faces, holemap_cells=cells, bin_cubes=bins)
    rf, rd, _, _ = O.cut(c.p, c.nodes, c.q, c.faces)
    check(f, d, rf, rd, 0.4)


def test_surface_outside_grid_and_grid_inside_surface():
    nodes = W.background(4, 2, jitter=0.05, seed=2)
    far = W.cubed_sphere(4, 2, radius=0.5, centre=(9.0, 9.0, 9.0))
    f, d, st = gpu_cut(2, nodes, 2, far)
    assert np.all(f == O.FIELD) and st["n_candidates"] == 0
    big = W.cubed_sphere(6, 2, radius=12.0, centre=(0.3, -0.2, 0.1))
    f, d, _ = gpu_cut(2, nodes, 2, big)
    rf, rd, _, _ = O.cut(2, nodes, 2, big)
    check(f, d, rf, rd, 1.0)
    assert np.all(f == O.HOLE)


def test_single_element_and_tiny_surface_inside_an_element():
    e = W.hex_block([0, 0, 0], [1, 1, 1], p=2)
    for F in (W.cubed_sphere(2, 2, radius=0.2, centre=(0.5, 0.45, 0.52)),      # inside the element
              W.cubed_sphere(2, 2, radius=0.6, centre=(0.5, 0.5, 0.5)),        # cutting through it
              W.cubed_sphere(2, 2, radius=3.0, centre=(0.5, 0.5, 0.5))):       # enclosing it
        f, d, _ = gpu_cut(2, e, 2, F)
        rf, rd, _, _ = O.cut(2, e, 2, F)
        check(f, d, rf, rd, 1.0)


def test_slot_and_concave_corner_surfaces():
    cells = [(x, y, z) for x in range(3) for y in range(2) for z in range(2) if not (x == 1 and y == 1)]
    F = W.polycube_surface(cells)
    nodes = np.concatenate([W.hex_block([1.25, 1.25, 0.25], [1.75, 1.75, 1.75], p=1, n=(1, 1, 3)),
                            W.hex_block([0.25, 0.25, 0.25], [0.75, 0.75, 0.75], p=1),
                            W.hex_block([-1.0, -1.0, -1.0], [4.0, 3.0, 3.0], p=1, n=(10, 8, 8))])
    f, d, _ = gpu_cut(1, nodes, 1, F)
    rf, rd, _, rst = O.cut(1, nodes, 1, F)
    assert rst["paper_rule_disagree"] == 0
    check(f, d, rf, rd, 0.5)
    L = W.polycube_surface([(0, 0, 0), (1, 0, 0), (0, 1, 0)])
    nodes = np.concatenate([W.hex_block([1.2, 1.2, 0.3], [1.6, 1.6, 0.7], p=2),
                            W.hex_block([-0.5, -0.5, -0.5], [2.5, 2.5, 1.5], p=2, n=(7, 7, 4))])
    f, d, _ = gpu_cut(2, nodes, 1, L)
    rf, rd, _, _ = O.cut(2, nodes, 1, L)
    check(f, d, rf, rd, 0.4)


def test_precisions_agree_and_repeat_bit_identically():
    c = W.dimpled_sphere_case(n=20, p=2, m=10, q=2, n_dimples=120, seed=8)
    f1, d1, s1 = gpu_cut(c.p, c.nodes, c.q, c.faces, precision=1)
    f2, d2, s2 = gpu_cut(c.p, c.nodes, c.q, c.faces, precision=0)
    f3, d3, _ = gpu_cut(c.p, c.nodes, c.q, c.faces, precision=1)
    assert np.array_equal(f1, f2) and np.array_equal(f1, f3)
    assert np.array_equal(d1, d3)
    fin = np.isfinite(d1)
    assert np.array_equal(fin, np.isfinite(d2))
    assert np.all(np.abs(d1[fin] - d2[fin]) <= 1e-12 * np.maximum(np.abs(d2[fin]), 0.2))
    assert s1["pairs_recheck"] < s1["pairs_bulk"]


GOLDEN64 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "scale64_cut.npz")


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


@pytest.mark.parametrize("form", ["flags_only_bench_shape", "flags_only_default_shape", "fp32_recheck_dist",
                                  "fp64_dist"])
def test_full_scale_dimpled_64cube_every_element(form):
    """The 262,144-element scale workload (64^3 Q2, sinusoidal curving, dimpled
    sphere of 6144 Q2 faces), every element against the oracle's stored cut:
    the flags-only form the benchmark times (its autotuned launch shape, 16
    warps per block, and the default shape), and both distance forms (FP32 bulk
    with FP64 re-solve, all FP64) with their distances."""
    c = W.dimpled_sphere_case()
    G = np.load(GOLDEN64)
    assert str(G["nodes_sha256"]) == _sha(c.nodes) and str(G["faces_sha256"]) == _sha(c.faces), \
        "the generated workload differs from the one the stored cut was computed on"
    assert int(G["undecidable"]) == 0
    ref_f = G["flags"]
    h = 4.0 / c.n
    dev = torch.device("cuda:0")
    tn = torch.from_numpy(c.nodes).to(dev)
    tf = torch.from_numpy(c.faces).to(dev)
    flags = torch.full((c.n_elem,), 7, dtype=torch.int8, device=dev)
    dist = None
    prec = dc.DC_FP64 if form == "fp64_dist" else dc.DC_FP32_RECHECK
    with dc.Context([(c.p, tn)], precision=prec) as ctx:
        if form == "flags_only_bench_shape":
            ctx.set_tuning(warps_per_cta=16, cands_per_warp=1)
        if form.endswith("_dist"):
            dist = torch.full((c.n_elem,), np.nan, dtype=torch.float64, device=dev)
        ctx.cut(0, c.q, tf, flags, dist)
        torch.cuda.synchronize()
        st = ctx.stats()
    f = flags.cpu().numpy()
    bad = np.nonzero(f != ref_f)[0]
    assert bad.size == 0, f"{bad.size} flag mismatches, first {bad[:8]}: gpu {f[bad[:8]]} oracle {ref_f[bad[:8]]}"
    if dist is None:
        return
    d = dist.cpu().numpy()
    assert not np.any(np.isnan(d))
    fin = np.nonzero(np.isfinite(d))[0]
    assert st["n_candidates"] == fin.size
    ids, rd = G["dist_ids"].astype(np.int64), G["dist"]
    pos = np.searchsorted(ids, fin)
    covered = (pos < ids.size) & (ids[np.minimum(pos, ids.size - 1)] == fin)
    assert covered.all(), f"{int((~covered).sum())} exact-test elements lie beyond the stored band"
    want = rd[pos]
    err = np.abs(d[fin] - want)
    assert np.all(err <= 1e-12 * np.maximum(np.abs(want), h)), f"max dist error {err.max():.3e}"
    # the hole map's elements: never fringe, side by the sign
    inf = ~np.isfinite(d)
    assert np.all(ref_f[inf] != O.FRINGE)
    assert np.array_equal(np.where(d[inf] > 0, O.FIELD, O.HOLE).astype(np.int8), ref_f[inf])


def test_fp32_stage_distances_are_reported_within_their_rounding_bound():
    """fp32_dist_out: the FP32 bulk's own distance of every exact-test element
    (before any FP64 re-solve) lies within the FP32 rounding bound of the
    final FP64 distance; hole-map elements get +-inf, elements the FP32 stage
    never measured NaN; the output is refused without dist_out or in the
    DC_FP64 precision."""
    c = W.dimpled_sphere_case(n=20, p=2, m=10, q=2, n_dimples=120, seed=8)
    dev = torch.device("cuda:0")
    tn = torch.from_numpy(c.nodes).to(dev)
    tf = torch.from_numpy(c.faces).to(dev)
    h = 4.0 / c.n
    f = torch.empty(c.n_elem, dtype=torch.int8, device=dev)
    d = torch.empty(c.n_elem, dtype=torch.float64, device=dev)
    d32 = torch.full((c.n_elem,), 7.0, dtype=torch.float32, device=dev)
    with dc.Context([(c.p, tn)], precision=dc.DC_FP32_RECHECK) as ctx:
        ctx.cut(0, c.q, tf, f, d, fp32_dist_out=d32)
        with pytest.raises(dc.DirectCutError) as ei:
            ctx.cut(0, c.q, tf, f, None, fp32_dist_out=d32)
        assert ei.value.status == dc.DC_EINVAL
        # host outputs take the same path through the arena's staging
        fh = np.empty(c.n_elem, dtype=np.int8)
        dh = np.empty(c.n_elem, dtype=np.float64)
        eh = np.full(c.n_elem, 7.0, dtype=np.float32)
        ctx.cut(0, c.q, c.faces, fh, dh, fp32_dist_out=eh)
    with dc.Context([(c.p, tn)], precision=dc.DC_FP64) as ctx:
        with pytest.raises(dc.DirectCutError) as ei:
            ctx.cut(0, c.q, tf, f, d, fp32_dist_out=d32)
        assert ei.value.status == dc.DC_EINVAL
    dd, ee = d.cpu().numpy(), d32.cpu().numpy()
    assert np.array_equal(ee, eh, equal_nan=True) and np.array_equal(dd, dh)
    fin = np.isfinite(dd)
    assert not np.any(ee == 7.0)
    assert np.array_equal(np.isinf(ee), ~fin)
    assert np.array_equal(np.sign(ee[~fin]), np.sign(dd[~fin]))
    have = fin & ~np.isnan(ee)
    assert have.sum() > 50
    # the same side, and within 64 u S (S < 2 h: element and nearby faces in
    # the element's frame)
    assert np.array_equal(np.signbit(ee[have]), np.signbit(dd[have]))
    assert np.all(np.abs(ee[have].astype(np.float64) - dd[have]) <= 64 * 2.0 ** -24 * 2 * h)
