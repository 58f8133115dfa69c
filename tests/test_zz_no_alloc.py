"""dc_cut_noalloc: the cut for callers that may not allocate device memory
when they cut -- real-time loops that forbid allocation after start-up
(cudaMalloc / cudaFree can block and synchronise the device) and hosts whose
own allocator owns the GPU's memory.  Its scratch is one fixed array inside the
library, shared by every call, so two calls in a row must each give the result
of the context path (dc_cut) and of the CPU oracle on their own input, with
and without distances.

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


class _FakeDeviceTensor:
    """Stands in for a CUDA tensor on a machine without one: the binding reads
    only its address, dtype and shape before it checks the shapes, and the
    shape checks come before any call into the library."""

    def __init__(self, shape, dtype):
        import torch
        self.shape = tuple(shape)
        self.dtype = dtype
        self.is_cuda = True
        self._torch = torch

    def data_ptr(self):
        return 256

    def is_contiguous(self):
        return True

    def dim(self):
        return len(self.shape)

    def numel(self):
        return int(np.prod(self.shape))


def test_noalloc_wrapper_rejects_wrong_shapes_before_calling_the_library():
    torch = pytest.importorskip("torch")
    dc = _lib()
    f64, i8 = torch.float64, torch.int8
    nodes = _FakeDeviceTensor((100, 27, 3), f64)
    faces = _FakeDeviceTensor((24, 9, 3), f64)
    flags = _FakeDeviceTensor((100,), i8)
    dist = _FakeDeviceTensor((100,), f64)
    bad = [
        dict(nodes=_FakeDeviceTensor((2700, 3), f64)),          # flattened nodes
        dict(nodes=_FakeDeviceTensor((100, 8, 3), f64)),        # p=1 nodes for p=2
        dict(faces=_FakeDeviceTensor((24, 4, 3), f64)),         # q=1 faces for q=2
        dict(flags_out=_FakeDeviceTensor((99,), i8)),           # short flags
        dict(dist_out=_FakeDeviceTensor((50,), f64)),           # short distances
    ]
    for kw in bad:
        args = dict(nodes=nodes, faces=faces, flags_out=flags, dist_out=dist)
        args.update(kw)
        with pytest.raises(ValueError):
            dc.dc_cut_noalloc(2, args["nodes"], 2, args["faces"], args["flags_out"], args["dist_out"])


@pytest.mark.gpu
def test_noalloc_matches_dc_cut_and_the_oracle_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle as O
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
            g_ref = torch.empty(case.n_elem, dtype=torch.int8, device=dev)
            ctx.cut(0, case.q, faces, g_ref, pose=pose)  # flags only (its own exact stage)
            f = torch.full((case.n_elem,), 9, dtype=torch.int8, device=dev)
            d = torch.full((case.n_elem,), np.nan, dtype=torch.float64, device=dev)
            dc.dc_cut_noalloc(case.p, nodes, case.q, faces, f, d, pose=pose)
            g = torch.full((case.n_elem,), 9, dtype=torch.int8, device=dev)
            dc.dc_cut_noalloc(case.p, nodes, case.q, faces, g, None, pose=pose)  # flags only
            torch.cuda.synchronize()
            fr, dr, gr = f_ref.cpu().numpy(), d_ref.cpu().numpy(), g_ref.cpu().numpy()
            fn, dn, gn = f.cpu().numpy(), d.cpu().numpy(), g.cpu().numpy()
            assert np.array_equal(fn, fr)
            assert np.array_equal(gn, fn)
            assert np.array_equal(gn, gr)
            fin = np.isfinite(dr)
            assert np.array_equal(fin, np.isfinite(dn))
            assert np.all(np.abs(dn[fin] - dr[fin]) <= 1e-12 * np.maximum(np.abs(dr[fin]), h))
            assert np.array_equal(np.sign(dn[~fin]), np.sign(dr[~fin]))
            # the oracle, every element: flags equal, distances where the
            # allocation-free cut computed them
            of, od, _, ost = O.cut(case.p, case.nodes, case.q, case.faces, pose=pose)
            assert ost["undecidable"] == 0
            assert np.array_equal(fn, of)
            fin = np.isfinite(dn)
            assert np.all(np.abs(dn[fin] - od[fin]) <= 1e-12 * np.maximum(np.abs(od[fin]), h))
