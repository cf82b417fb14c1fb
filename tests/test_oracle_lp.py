"""Pins of the oracle's moment conditions and phase-I simplex (Sec. 2, 3.2,
3.6, 4.1).

* Brute force: vertex enumeration over every m-column basis of a tiny
  neighbourhood gives the exact feasibility verdict, and the oracle's answer
  must be one of those vertices.
* Lemma fnorm: 4 (R)^-2 <= sum f~ <= 4 (r)^-2, i.e. 1 <= sum f~ <= 16 for
  r = 1/2, R = 2, and sum f~ = 4/rho^2 when every neighbour sits at rho.
* Sec. 3.6: adding the |alpha| = 4 condition sum f |xi|^4 = 0 makes every
  neighbourhood infeasible.
"""
import itertools
import math

import numpy as np
import pytest

B5 = np.array([0.0, 0.0, 2.0, 0.0, 2.0])


def textbook_vandermonde(xi, eta):
    # rows (1,0) (0,1) (2,0) (1,1) (0,2): r^alpha with r in units of h
    return np.array([xi, eta, xi ** 2, xi * eta, eta ** 2])


def vertices(V, b, tol=1e-9):
    m, K = V.shape
    out = []
    for S in itertools.combinations(range(K), m):
        A = V[:, S]
        if abs(np.linalg.det(A)) < 1e-10:
            continue
        fs = np.linalg.solve(A, b)
        if (fs >= -tol).all():
            f = np.zeros(K)
            f[list(S)] = np.maximum(fs, 0)
            out.append(f)
    return out


def ring(rng, K, lo=0.5, hi=2.0, arc=2 * np.pi):
    th = rng.uniform(0, arc, K)
    rad = np.sqrt(rng.uniform(lo * lo, hi * hi, K))
    return rad * np.cos(th), rad * np.sin(th)


def test_vandermonde_rows_match_multi_indices(orc):
    rng = np.random.default_rng(5)
    xi, eta = ring(rng, 9)
    V = orc.vandermonde(1, xi, eta)
    np.testing.assert_array_equal(V, textbook_vandermonde(xi, eta))
    V2 = orc.vandermonde(2, xi, eta)
    np.testing.assert_allclose(V2[5:], np.array([xi ** 3, xi ** 2 * eta, xi * eta ** 2, eta ** 3]), rtol=1e-15)


@pytest.mark.parametrize("seed", range(60))
def test_phase1_agrees_with_vertex_enumeration(orc, seed):
    rng = np.random.default_rng(100 + seed)
    K = int(rng.integers(5, 11))
    arc = 2 * np.pi if seed % 4 else rng.uniform(np.pi * 0.6, np.pi * 1.2)
    xi, eta = ring(rng, K, arc=arc)
    V = textbook_vandermonde(xi, eta)
    st, f, npiv, res = orc.phase1(V, B5)
    verts = vertices(V, B5)
    if not verts:
        assert st != 0
        return
    assert st == 0, "feasible by enumeration but oracle says %d" % st
    assert res <= 1e-12  # random clouds give non-degenerate vertices
    assert (f >= 0).all()
    np.testing.assert_allclose(V @ f, B5, atol=1e-12)
    assert np.count_nonzero(f) <= 5
    assert min(np.max(np.abs(f - v)) for v in verts) < 1e-9


def test_phase1_infeasible_half_plane(orc):
    # all neighbours on one side: sum f xi = 0 forces f = 0 (Sec. 4.2 motive)
    rng = np.random.default_rng(7)
    xi = rng.uniform(0.5, 2.0, 8)
    eta = rng.uniform(-1, 1, 8)
    st, f, _, _ = orc.phase1(textbook_vandermonde(xi, eta), B5)
    assert st == 1 and not f.any()


@pytest.mark.parametrize("seed", range(40))
def test_lemma_fnorm_bounds(orc, seed):
    rng = np.random.default_rng(200 + seed)
    xi, eta = ring(rng, 8 + seed % 9)
    st, f, _, _ = orc.phase1(textbook_vandermonde(xi, eta), B5)
    if st == 0:
        s = f.sum()
        assert 1.0 - 1e-12 <= s <= 16.0 + 1e-12
        # sum f |xi|^2 = 4 (sum of the (2,0) and (0,2) rows)
        assert abs(np.sum(f * (xi ** 2 + eta ** 2)) - 4.0) < 1e-12


@pytest.mark.parametrize("rho", [0.5, 0.8, 1.0, 1.5, 2.0])
def test_equidistant_sum(orc, rho):
    rng = np.random.default_rng(int(rho * 10))
    th = rng.uniform(0, 2 * np.pi) + np.arange(8) * np.pi / 4
    xi, eta = rho * np.cos(th), rho * np.sin(th)
    st, f, _, _ = orc.phase1(textbook_vandermonde(xi, eta), B5)
    assert st == 0
    assert abs(f.sum() - 4.0 / rho ** 2) < 1e-12 * 16


def test_five_point_stencil_on_lattice_axes(orc):
    # the four axis neighbours at distance 1 carry the classical five-point
    # stencil f~ = 1 (Sec. 3.3 remark); with them first in column order the
    # phase-I vertex found is that stencil
    xi = np.array([1.0, 0.0, -1.0, 0.0, 1.0, -1.0, -1.0, 1.0])
    eta = np.array([0.0, 1.0, 0.0, -1.0, 1.0, 1.0, -1.0, -1.0])
    st, f, _, _ = orc.phase1(textbook_vandermonde(xi, eta), B5)
    assert st == 0
    np.testing.assert_allclose(f, [1, 1, 1, 1, 0, 0, 0, 0], atol=1e-14)


@pytest.mark.parametrize("seed", range(20))
def test_fourth_order_conditions_infeasible(orc, seed):
    # Sec. 3.6: sum_j f_ij |r_ij|^4 = 0 with f >= 0 forces f = 0, which
    # contradicts the |alpha| = 2 rows
    rng = np.random.default_rng(300 + seed)
    xi, eta = ring(rng, 12)
    V = np.vstack([textbook_vandermonde(xi, eta), (xi ** 2 + eta ** 2) ** 2])
    b = np.concatenate([B5, [0.0]])
    st, f, _, _ = orc.phase1(V, b)
    assert st == 1


def test_degenerate_inputs(orc):
    # fewer columns than rows and no columns at all are infeasible, not errors
    st, f, _, _ = orc.phase1(np.zeros((5, 0)), B5)
    assert st == 1
    rng = np.random.default_rng(9)
    xi, eta = ring(rng, 3)
    st, f, _, _ = orc.phase1(textbook_vandermonde(xi, eta), B5)
    assert st == 1


# Four axis neighbours at distance 1 meet every moment condition with
# weights 1 (the five-point stencil).  Moving the one on +eta by eps < 0
# along xi breaks the (1,1) row, and the fifth column (0.7, 0.9) takes the
# weight -eps/0.63 to restore it: the unique solution on these five columns.
# For eps = -2e-12 and -5e-12 that weight (3.2e-12, 7.9e-12) is below the
# snap threshold 1e-11, so the vertex comes out with it set to zero and a
# moment residual of 0.9 * 3.2e-12 and 0.9 * 7.9e-12: above 1e-12, the LP is
# rejected (the moment conditions must hold to 1e-12 per particle).  For
# eps = -8e-12 the weight 1.27e-11 is kept and the residual is at rounding
# level.
SNAP_CASES = [(-2e-12, 1), (-5e-12, 1), (-8e-12, 0), (-2e-11, 0)]


def snap_columns(eps):
    return np.array([1.0, -1.0, eps, 0.0, 0.7]), np.array([0.0, 0.0, 1.0, -1.0, 0.9])


@pytest.mark.parametrize("eps,verdict", SNAP_CASES)
def test_residual_bar_is_1e12_after_snapping(orc, eps, verdict):
    xi, eta = snap_columns(eps)
    V = textbook_vandermonde(xi, eta)
    exact = np.linalg.solve(V, B5)
    assert np.all(exact > 0)
    assert abs(exact[4] - (-eps / 0.63)) <= 1e-3 * abs(eps)
    st, f, npiv, res = orc.phase1(V, B5)
    assert st == verdict, (st, res)
    if verdict == 0:
        np.testing.assert_allclose(f, exact, rtol=1e-9)
        assert res <= 1e-15
    else:
        # the residual the snapped vertex would leave
        snapped = np.where(exact > 1e-11, exact, 0.0)
        assert np.max(np.abs(V @ snapped - B5)) > 1e-12
        assert not f.any()
