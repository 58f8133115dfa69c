"""dc_cut_noalloc: the cut for callers that cannot allocate device memory when
they cut (stream capture, allocation-free real-time loops, hosts that own all
device memory).  Its scratch is one fixed array inside the library, shared by
every call, so two calls in a row must each match dc_cut on its own input.
This file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import workloads as W


def _lib():
    import paper_1711_07663_gb300 as dc
    from paper_1711_07663_gb300 import build as B
    B.build()
    dc.load()
    return dc


def test_noalloc_rejects_sizes_beyond_its_array():
    dc = _lib()
    fake = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    st = dc.load().dc_cut_noalloc(2, 10_000_000, fake, 2, 100, fake, None, 0.0, fake, None, None)
    assert st == dc.DC_EINVAL
    assert "scratch" in dc.dc_last_error()


@pytest.mark.gpu
def test_noalloc_matches_dc_cut_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dc = _lib()
    dev = torch.device("cuda:0")
    case = W.dimpled_sphere_case(n=16, p=2, m=8, q=2, n_dimples=60, seed=31)
    nodes = torch.from_numpy(case.nodes).to(dev)
    faces = torch.from_numpy(case.faces).to(dev)
    poses = [None, np.concatenate([W.random_rotation(W.rng(4)), np.array([[0.05], [-0.08], [0.02]])], axis=1)]
    h = 4.0 / case.n
    # the same hole-map resolution as the allocation-free cut (64 cubes), so
    # that the same elements are settled by the map (their distances are +-inf)
    with dc.Context([(case.p, nodes)], holemap_cells=64) as ctx:
        for pose in poses:  # two calls in a row share the library's scratch array
            f_ref = torch.empty(case.n_elem, dtype=torch.int8, device=dev)
            d_ref = torch.empty(case.n_elem, dtype=torch.float64, device=dev)
            ctx.cut(0, case.q, faces, f_ref, d_ref, pose=pose)
            f = torch.full((case.n_elem,), 9, dtype=torch.int8, device=dev)
            d = torch.full((case.n_elem,), np.nan, dtype=torch.float64, device=dev)
            dc.dc_cut_noalloc(case.p, nodes, case.q, faces, f, d, pose=pose)
            torch.cuda.synchronize()
            fr, dr, fn, dn = f_ref.cpu().numpy(), d_ref.cpu().numpy(), f.cpu().numpy(), d.cpu().numpy()
            assert np.array_equal(fn, fr)
            fin = np.isfinite(dr)
            assert np.array_equal(fin, np.isfinite(dn))
            assert np.all(np.abs(dn[fin] - dr[fin]) <= 1e-12 * np.maximum(np.abs(dr[fin]), h))
            assert np.array_equal(np.sign(dn[~fin]), np.sign(dr[~fin]))
