"""Allocation failures.  Every device and pinned-host allocation the library
makes can be made to fail on purpose (dc_fail_alloc, host side: the allocation
reports failure without being attempted).  For each allocation of a fixed
sequence of calls in turn, the call that meets the failure must return
DC_ENOMEM, and once the failure is disarmed the same context (or, when
dc_create failed, a new one) must finish the sequence with the results of a
run without failures.  No device memory may be left behind."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _dc():
    import paper_1711_07663_gb300 as dc
    from paper_1711_07663_gb300 import build as B
    B.build()
    dc.load()
    return dc


def _steps(dc, case, big, reserve, out):
    """The sequence: create, a host cut, a host cut with distances, a submit
    with distances (and its poll), a cut with a larger surface, a donor search.
    Each step stores what it computed in `out`."""
    st = {}

    def create():
        st["ctx"] = dc.Context([(case.p, case.nodes)], reserve_faces=reserve)

    def cut():
        out["flags"] = st["ctx"].cut(0, case.q, case.faces)

    def cut_dist():
        d = np.empty(case.n_elem)
        out["flags_d"] = st["ctx"].cut(0, case.q, case.faces, dist_out=d)
        out["dist"] = d

    def submit():
        f = np.empty(case.n_elem, dtype=np.int8)
        d = np.empty(case.n_elem)
        t = st["ctx"].submit(0, case.q, case.faces, f, d)
        assert st["ctx"].poll(t, timeout_us=-1) == 0
        out["flags_s"], out["dist_s"] = f, d

    def cut_big():
        out["flags_big"] = st["ctx"].cut(0, big.q, big.faces)

    def locate():
        pl = dc.PointLocator(case.p, case.nodes)
        try:
            pts = W.shell_points(2000, 0.5, 1.5, seed=5)
            out["donor"], out["ref"] = pl.locate(pts)
        finally:
            pl.close()

    return st, [create, cut, cut_dist, submit, cut_big, locate]


def _run(dc, case, big, reserve, fail_at=None):
    """Run the sequence, with the allocation `fail_at` allocations after the
    start made to fail.  Returns (results, allocations made, the failed step)."""
    out = {}
    st, steps = _steps(dc, case, big, reserve, out)
    n0 = dc.dc_fail_alloc(-1 if fail_at is None else fail_at)
    failed = None
    try:
        i = 0
        while i < len(steps):
            try:
                steps[i]()
            except dc.DirectCutError as e:
                assert fail_at is not None and failed is None, (steps[i].__name__, e)
                assert e.status == dc.DC_ENOMEM, (steps[i].__name__, e)
                failed = steps[i].__name__
                dc.dc_fail_alloc(-1)
                continue  # the same step once more, memory now available
            i += 1
    finally:
        n1 = dc.dc_fail_alloc(-1)
        if "ctx" in st:
            st["ctx"].close()
    return out, n1 - n0, failed


@pytest.mark.parametrize("reserve", [0, -1], ids=["reserved_arenas", "lazy_arenas"])
def test_every_allocation_failure_is_reported_and_recovered(reserve):
    dc = _dc()
    import torch
    case = W.sphere_in_box(n=16, m=8)
    big = W.sphere_in_box(n=16, m=24)
    ref, n_alloc, failed = _run(dc, case, big, reserve)
    assert failed is None and n_alloc >= 4
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    seen = set()
    for k in range(n_alloc):
        got, _, failed = _run(dc, case, big, reserve, fail_at=k)
        assert failed is not None, f"allocation {k} of {n_alloc} did not fail any call"
        seen.add(failed)
        for key, val in ref.items():
            assert np.array_equal(got[key], val), (k, failed, key)
    assert "create" in seen
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    # the library frees what a failed call held: n_alloc failing runs leave
    # no more than allocator rounding behind
    assert free0 - free1 < 32 << 20, (free0, free1, n_alloc)
