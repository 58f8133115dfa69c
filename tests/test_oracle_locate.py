"""Pins of the oracle's donor search (point connectivity, Eqs. reftophys,
ref-update): the Lagrange basis against its defining properties and finite
differences, the isoparametric map and Newton against the closed-form inverse
of affine elements, recovery of generated points inside curved elements,
rigid-motion invariance, points outside the grid, and the lowest-index rule on
shared faces."""
import numpy as np
import pytest

import oracle as O
import workloads as W


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lagrange_basis(p):
    nodes = -1.0 + 2.0 * np.arange(p + 1) / p
    for j, x in enumerate(nodes):
        l, _ = O.lagrange(p, x)
        assert np.allclose(l, np.eye(p + 1)[j], atol=1e-14)
    for x in np.linspace(-1.2, 1.2, 13):
        l, dl = O.lagrange(p, x)
        assert abs(l.sum() - 1.0) < 1e-13 and abs(dl.sum()) < 1e-12
        # exact on polynomials of degree <= p, and their derivatives
        for k in range(p + 1):
            assert abs((nodes ** k * l).sum() - x ** k) < 1e-12
            assert abs((nodes ** k * dl).sum() - (k * x ** (k - 1) if k else 0.0)) < 1e-11
        e = 1e-6
        fd = (O.lagrange(p, x + e)[0] - O.lagrange(p, x - e)[0]) / (2 * e)
        assert np.allclose(dl, fd, atol=1e-7)


def affine_element(p, x0, A):
    """Order-p element of the affine map x = x0 + A xi (nodes at the
    equispaced reference points)."""
    r = -1.0 + 2.0 * np.arange(p + 1) / p
    out = np.zeros(((p + 1) ** 3, 3))
    for k in range(p + 1):
        for j in range(p + 1):
            for i in range(p + 1):
                out[i + (p + 1) * (j + (p + 1) * k)] = x0 + A @ np.array([r[i], r[j], r[k]])
    return out


@pytest.mark.parametrize("p", [1, 2, 3])
def test_map_and_newton_on_affine_elements(p):
    g = np.random.default_rng(p)
    for _ in range(5):
        A = g.normal(size=(3, 3)) * 0.3 + np.eye(3) * 0.5
        x0 = g.normal(size=3)
        en = affine_element(p, x0, A)
        for _ in range(5):
            xi = g.uniform(-0.95, 0.95, size=3)
            x, J = O.iso_map(p, en, xi)
            assert np.allclose(x, x0 + A @ xi, atol=1e-13)
            assert np.allclose(J, A, atol=1e-12)
            # affine map: one Newton step from 0 lands on the closed form
            ok, got, res, it = O.newton(p, en, x0 + A @ xi, 1.0)
            assert ok and it == 1
            assert np.allclose(got, np.linalg.solve(A, (x0 + A @ xi) - x0), atol=1e-12)


def test_points_generated_inside_curved_elements_are_recovered():
    nodes = W.sphere_shell(5, 3, 2, 1.0, 1.6)
    g = np.random.default_rng(7)
    E = g.integers(0, nodes.shape[0], size=300)
    xs = g.uniform(-0.97, 0.97, size=(300, 3))
    pts = np.array([O.iso_map(2, nodes[e], x)[0] for e, x in zip(E, xs)])
    donor, ref, m = O.locate(2, nodes, pts)
    assert np.array_equal(donor, E)
    assert np.abs(ref - xs).max() < 1e-8
    # the returned reference point maps back onto the point
    back = np.array([O.iso_map(2, nodes[e], x)[0] for e, x in zip(donor, ref)])
    assert np.abs(back - pts).max() < 1e-10
    assert np.all(m[:, 0] >= 0) and np.all(m[:, 1] > 0)


def test_points_outside_the_grid_have_no_donor():
    nodes = W.sphere_shell(4, 2, 2, 1.0, 1.6)
    g = np.random.default_rng(8)
    d = g.normal(size=(100, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    inner = d[:50] * g.uniform(0.2, 0.9, size=(50, 1))
    outer = d[50:] * g.uniform(1.75, 3.0, size=(50, 1))
    donor, _, _ = O.locate(2, nodes, np.concatenate([inner, outer]))
    assert np.all(donor == -1)


def test_rigid_motion_of_grid_and_points():
    nodes = W.sphere_shell(4, 2, 2, 1.0, 1.6)
    pts = W.shell_points(200, 1.02, 1.58, seed=3)
    d0, r0, _ = O.locate(2, nodes, pts)
    R = W.axis_rotation([0.3, -0.5, 0.8], 0.7)
    t = np.array([0.25, -0.5, 1.0])
    pose = np.concatenate([R, t[:, None]], axis=1)
    d1, r1, _ = O.locate(2, nodes, pts @ R.T + t, pose=pose)
    assert np.array_equal(d0, d1)
    assert np.abs(r0 - r1).max() < 1e-8
    assert (d0 >= 0).mean() > 0.95


def test_shared_face_takes_the_lowest_index():
    # two unit cubes sharing the face x = 1
    a = affine_element(2, np.array([0.5, 0.5, 0.5]), 0.5 * np.eye(3))
    b = affine_element(2, np.array([1.5, 0.5, 0.5]), 0.5 * np.eye(3))
    pts = np.array([[1.0, 0.3, 0.6], [1.0, 0.9, 0.2], [0.999, 0.5, 0.5], [1.001, 0.5, 0.5]])
    donor, ref, _ = O.locate(2, np.stack([a, b]), pts)
    assert donor.tolist() == [0, 0, 0, 1]
    donor, ref, _ = O.locate(2, np.stack([b, a]), pts)
    assert donor.tolist() == [0, 0, 1, 0]
    assert np.allclose(ref[0], [-1.0, -0.4, 0.2], atol=1e-12)
