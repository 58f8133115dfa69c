"""Pins for the oracle's triangle-triangle distance (the primitive of the
modified Moller test, Sec. 4.2 / Alg. cp1 and cp2 of the paper).

Each pin is independent of the oracle's own decomposition:
  * exact rational arithmetic by active-set enumeration of the convex QP
    min |sum l_i A_i - sum m_j B_j|^2 over the two simplices,
  * closed-form configurations,
  * dense barycentric sampling (an upper bound converging from above),
  * invariances (symmetry, vertex order, exact power-of-two scaling).
"""
import itertools
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

getcontext().prec = 50


# ---------------------------------------------------------------- exact QP
def _solve(G, r):
    """Gaussian elimination over the rationals; None when singular."""
    n = len(r)
    M = [list(G[i]) + [r[i]] for i in range(n)]
    for c in range(n):
        piv = next((i for i in range(c, n) if M[i][c] != 0), None)
        if piv is None:
            return None
        M[c], M[piv] = M[piv], M[c]
        for i in range(n):
            if i != c and M[i][c] != 0:
                f = M[i][c] / M[c][c]
                M[i] = [a - f * b for a, b in zip(M[i], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)]


def _dot(a, b):
    return sum(x * y for x, y in zip(a, b))


def exact_d2(A, B):
    """Squared distance between conv(A) and conv(B) (3 points each, rational
    coordinates), exact: the optimum with minimal support solves the
    equality-constrained normal equations on the affine hulls of its faces."""
    A = [[Fraction(v) for v in p] for p in A]
    B = [[Fraction(v) for v in p] for p in B]
    subsets = [s for r in (1, 2, 3) for s in itertools.combinations(range(3), r)]
    best = None
    for I in subsets:
        for J in subsets:
            base = [A[I[0]][k] - B[J[0]][k] for k in range(3)]
            dirs = [[A[i][k] - A[I[0]][k] for k in range(3)] for i in I[1:]]
            dirs += [[-(B[j][k] - B[J[0]][k]) for k in range(3)] for j in J[1:]]
            m = len(dirs)
            x = []
            if m:
                G = [[_dot(di, dj) for dj in dirs] for di in dirs]
                rhs = [-_dot(di, base) for di in dirs]
                x = _solve(G, rhs)
                if x is None:
                    continue
            nl = len(I) - 1
            lam = [1 - sum(x[:nl])] + x[:nl]
            mu = [1 - sum(x[nl:])] + x[nl:]
            if any(v < 0 for v in lam + mu):
                continue
            diff = [base[k] + sum(x[t] * dirs[t][k] for t in range(m)) for k in range(3)]
            d2 = _dot(diff, diff)
            if best is None or d2 < best:
                best = d2
    return best


def _sqrt_float(fr):
    return float((Decimal(fr.numerator) / Decimal(fr.denominator)).sqrt())


@pytest.mark.parametrize("seed", range(6))
def test_tritri_matches_exact_rational(seed):
    g = np.random.default_rng(seed)
    for _ in range(25):
        A = g.integers(-6, 7, size=(3, 3))
        B = g.integers(-6, 7, size=(3, 3))
        # bias half the cases into near-touching / crossing placements
        if g.random() < 0.5:
            B = B // 2 + A[g.integers(0, 3)] // 2
        d2 = exact_d2(A.tolist(), B.tolist())
        d_exact = _sqrt_float(d2)
        d, ca, cb = O.tritri(A.astype(float), B.astype(float))
        assert abs(d - d_exact) <= 4e-15 * max(1.0, d_exact), (A, B, d, d_exact)
        # the returned closest points realise the distance and lie on the triangles
        assert abs(np.linalg.norm(ca - cb) - d) <= 1e-12 * max(1.0, d)


def test_exact_qp_itself_on_known_cases():
    # two unit triangles stacked 3 apart along z
    A = [[0, 0, 0], [1, 0, 0], [0, 1, 0]]
    B = [[0, 0, 3], [1, 0, 3], [0, 1, 3]]
    assert exact_d2(A, B) == 9
    # crossing
    B = [[Fraction(1, 4), Fraction(1, 4), -1], [Fraction(1, 4), Fraction(1, 4), 1], [5, 5, 0]]
    assert exact_d2(A, B) == 0


# ---------------------------------------------------------------- closed forms
def test_parallel_offset_triangles():
    T = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    for h in (1e-9, 1e-3, 0.5, 7.25):
        d, _, _ = O.tritri(T, T + [0.0, 0.0, h])
        assert d == pytest.approx(h, rel=1e-14, abs=1e-300)


def test_coplanar_gap():
    A = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    B = np.array([[1.5, 0.0, 0.0], [3.0, 0.0, 0.0], [1.5, 1.0, 0.0]])
    d, _, _ = O.tritri(A, B)
    assert d == pytest.approx(0.5, rel=1e-15)


def test_crossing_is_zero():
    A = np.array([[0.0, 0.0, 0.0], [4.0, 0.0, 0.0], [0.0, 4.0, 0.0]])
    B = np.array([[1.0, 1.0, -1.0], [1.0, 1.0, 1.0], [2.0, 0.5, 1.0]])
    d, ca, cb = O.tritri(A, B)
    assert d == 0.0
    assert np.allclose(ca, [1.0, 1.0, 0.0])


def test_vertex_over_face():
    A = np.array([[0.0, 0.0, 0.0], [4.0, 0.0, 0.0], [0.0, 4.0, 0.0]])
    B = np.array([[1.0, 1.0, 0.3], [1.0, 5.0, 9.0], [6.0, 1.0, 9.0]])
    d, ca, cb = O.tritri(A, B)
    assert d == pytest.approx(0.3, rel=1e-14)
    assert np.allclose(ca, [1.0, 1.0, 0.0]) and np.allclose(cb, [1.0, 1.0, 0.3])


def test_skew_edges():
    # edge of A along x at z=0, edge of B along y at z=h, crossing over (1,1)
    h = 0.375
    A = np.array([[0.0, 1.0, 0.0], [2.0, 1.0, 0.0], [1.0, 1.0, -5.0]])
    B = np.array([[1.0, 0.0, h], [1.0, 2.0, h], [1.0, 1.0, h + 5.0]])
    d, ca, cb = O.tritri(A, B)
    assert d == pytest.approx(h, rel=1e-14)
    assert np.allclose(ca, [1.0, 1.0, 0.0]) and np.allclose(cb, [1.0, 1.0, h])


def test_segment_distance_closed_forms():
    # skew perpendicular segments
    d, _, _ = O.seg_seg([0, 0, 0], [2, 0, 0], [1, -1, 3], [1, 1, 3])
    assert d == pytest.approx(3.0)
    # parallel overlapping
    d, _, _ = O.seg_seg([0, 0, 0], [2, 0, 0], [1, 0.5, 0], [3, 0.5, 0])
    assert d == pytest.approx(0.5)
    # collinear disjoint
    d, _, _ = O.seg_seg([0, 0, 0], [1, 0, 0], [3, 0, 0], [4, 0, 0])
    assert d == pytest.approx(2.0)


def test_point_triangle_regions():
    T = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    assert O.pt_tri([0.2, 0.2, 0.7], T)[0] == pytest.approx(0.7)          # face
    assert O.pt_tri([-1.0, -1.0, 0.0], T)[0] == pytest.approx(np.sqrt(2))  # vertex
    assert O.pt_tri([0.5, -2.0, 0.0], T)[0] == pytest.approx(2.0)         # edge


# ---------------------------------------------------------------- sampling
def _bary_samples(T, n):
    pts = []
    for i in range(n + 1):
        for j in range(n + 1 - i):
            a, b = i / n, j / n
            pts.append(T[0] + a * (T[1] - T[0]) + b * (T[2] - T[0]))
    return np.array(pts)


@pytest.mark.parametrize("seed", range(4))
def test_tritri_against_dense_sampling(seed):
    g = np.random.default_rng(100 + seed)
    n = 48
    for _ in range(6):
        A = g.normal(size=(3, 3))
        B = g.normal(size=(3, 3)) + g.normal(size=3) * 0.7
        d, _, _ = O.tritri(A, B)
        PA, PB = _bary_samples(A, n), _bary_samples(B, n)
        dm = np.sqrt(((PA[:, None, :] - PB[None, :, :]) ** 2).sum(-1)).min()
        size = max(np.ptp(A, axis=0).max(), np.ptp(B, axis=0).max())
        assert d <= dm + 1e-12
        assert dm <= d + 2.0 * size / n


# ---------------------------------------------------------------- invariances
@pytest.mark.parametrize("seed", range(3))
def test_invariances(seed):
    g = np.random.default_rng(200 + seed)
    for _ in range(40):
        A = np.round(g.normal(size=(3, 3)) * 1024) / 1024
        B = np.round((g.normal(size=(3, 3)) + g.normal(size=3)) * 1024) / 1024
        d, _, _ = O.tritri(A, B)
        assert O.tritri(B, A)[0] == pytest.approx(d, rel=1e-14, abs=1e-15)
        for perm in itertools.permutations(range(3)):
            assert O.tritri(A[list(perm)], B[::-1])[0] == pytest.approx(d, rel=1e-14, abs=1e-15)
        # power-of-two scaling is exact in every operation
        assert O.tritri(A * 8.0, B * 8.0)[0] == 8.0 * d
        assert O.tritri(A * 0.25, B * 0.25)[0] == 0.25 * d
        t = np.array([32.0, -64.0, 16.0])
        assert O.tritri(A + t, B + t)[0] == pytest.approx(d, rel=1e-12, abs=1e-13)
