"""The autotuner and the launch shapes it sweeps, on the GPU through the C ABI:
no setting changes a flag (each matches the FP64 oracle), the tuner picks a
setting of its sweep and leaves it on the context, and bad settings are
refused without changing the current one."""
import itertools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
dc = None

CPE = (1.2, 1.8, 2.7)
BINS = (2, 4, 8)
WARPS = (4, 8, 16)
CPW = (1, 2, 4, 8)


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


def test_every_setting_gives_the_oracle_flags():
    c = W.sphere_in_box(n=16, p=2, m=8, q=2, seed=1)
    want, _, _, _ = O.cut(c.p, c.nodes, c.q, c.faces)
    with dc.Context([(c.p, c.nodes)]) as ctx:
        default = ctx.tuning()
        assert (round(default["cubes_per_edge"], 3), default["bin_cubes"], default["warps_per_cta"],
                default["cands_per_warp"]) == (1.8, 4, 8, 1)
        for cpe, bc, wpc, cpw in itertools.product(CPE, BINS, WARPS, CPW):
            ctx.set_tuning(cubes_per_edge=cpe, bin_cubes=bc, warps_per_cta=wpc, cands_per_warp=cpw)
            got = ctx.cut(0, c.q, c.faces)
            assert np.array_equal(got, want), (cpe, bc, wpc, cpw)


def test_autotune_on_a_ragged_batch():
    cases = W.batch_cases(count=8, seed=5, n_range=(8, 16), m_choices=(8, 16))
    meshes = [(cs.p, cs.nodes) for cs in cases]
    outs = [np.full(cs.n_elem, 9, dtype=np.int8) for cs in cases]
    reqs = [dict(q=cs.q, faces=cs.faces, flags_out=o, pose=cs.pose) for cs, o in zip(cases, outs)]
    with dc.Context(meshes) as ctx:
        best, trials = ctx.autotune(list(range(len(cases))), reqs, repeats=2)
        assert trials == len(CPE) * len(BINS) * len(WARPS) * len(CPW)
        assert best["ms"] > 0
        key = (round(best["cubes_per_edge"], 3), best["bin_cubes"], best["warps_per_cta"], best["cands_per_warp"])
        assert key[0] in CPE and key[1:] in set(itertools.product(BINS, WARPS, CPW))
        now = ctx.tuning()
        assert (round(now["cubes_per_edge"], 3), now["bin_cubes"], now["warps_per_cta"], now["cands_per_warp"]) == key
    for cs, f in zip(cases, outs):
        want, _, _, _ = O.cut(cs.p, cs.nodes, cs.q, cs.faces, pose=cs.pose)
        assert np.array_equal(f, want), cs.name


def test_a_fixed_hole_map_sweeps_only_launch_shapes():
    c = W.sphere_in_box(n=12, p=2, m=8, q=2, seed=4)
    want, _, _, _ = O.cut(c.p, c.nodes, c.q, c.faces)
    out = np.empty(c.n_elem, dtype=np.int8)
    with dc.Context([(c.p, c.nodes)], holemap_cells=48) as ctx:
        best, trials = ctx.autotune([0], [dict(q=c.q, faces=c.faces, flags_out=out)], repeats=1)
    assert trials == len(BINS) * len(WARPS) * len(CPW)
    assert abs(best["cubes_per_edge"] - 1.8) < 1e-6
    assert np.array_equal(out, want)


@pytest.mark.parametrize("bad", [dict(cubes_per_edge=0.4), dict(cubes_per_edge=4.5), dict(cubes_per_edge=float("nan")),
                                 dict(bin_cubes=1), dict(bin_cubes=17), dict(warps_per_cta=6),
                                 dict(warps_per_cta=32), dict(cands_per_warp=3), dict(cands_per_warp=0)])
def test_bad_settings_are_refused(bad):
    c = W.sphere_in_box(n=4, p=1, m=2, q=1, seed=2)
    with dc.Context([(c.p, c.nodes)]) as ctx:
        before = ctx.tuning()
        with pytest.raises(dc.DirectCutError) as ei:
            ctx.set_tuning(**bad)
        assert ei.value.status == -1
        assert ctx.tuning() == before
