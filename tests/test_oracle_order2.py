"""Pins of the oracle's n = 2 variant (Sec. 2, Eqs. cond_two, cond_alpha:
m = 9 moment rows, the cubic monomials added).

* Brute force: vertex enumeration over every 9-column basis of a tiny
  neighbourhood gives the exact feasibility verdict for the nine rows, and
  the oracle's answer must be one of those vertices.
* Polynomial exactness: a stencil that meets the nine conditions applies the
  Laplacian exactly to every polynomial of degree <= 3 (the Taylor argument of
  Sec. 2); an n = 1 stencil does not, in general, for the cubic ones.
* Order of consistency: on jittered clouds the operator's error on a smooth
  field falls like h^2 for n = 2 and like h for n = 1 (O(h^n), Sec. 2).
* Symmetry: on a lattice the classical five-point stencil meets every odd
  moment, so the small neighbourhood is feasible for n = 2 as well.
* Storage: a basic solution has up to 9 nonzero weights, all of them kept.
* Growth control: the step leaves out the longest prefix within
  C_diff h^4 ||Gamma||_1 (Eq. reduced_bound with n = 2), found here by brute
  force with exact rational sums.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import vrm_inputs

B9 = np.array([0.0, 0.0, 2.0, 0.0, 2.0, 0.0, 0.0, 0.0, 0.0])

# the ten monomials xi^a eta^b of degree <= 3 with their Laplacians at 0
MONOMIALS = [(a, b) for a in range(4) for b in range(4) if a + b <= 3]


def lap_at_zero(a, b):
    # Laplacian of xi^a eta^b at the origin: 2 for xi^2 and eta^2, else 0
    return 2.0 if (a, b) in ((2, 0), (0, 2)) else 0.0


def textbook_vandermonde9(xi, eta):
    return np.array([xi, eta, xi ** 2, xi * eta, eta ** 2, xi ** 3, xi ** 2 * eta, xi * eta ** 2, eta ** 3])


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


def symmetric_ring(rng, K, jitter):
    # K/2 points and their mirror images through the centre, then jittered:
    # near point symmetry keeps the odd moments within reach
    half = K // 2
    th = rng.uniform(0, 2 * np.pi, half)
    rad = np.sqrt(rng.uniform(0.25, 4.0, half))
    xi = np.concatenate([rad * np.cos(th), -rad * np.cos(th)])
    eta = np.concatenate([rad * np.sin(th), -rad * np.sin(th)])
    xi = xi + rng.uniform(-jitter, jitter, xi.size)
    eta = eta + rng.uniform(-jitter, jitter, eta.size)
    return xi, eta


def jitter_of(seed):
    return 0.05 * (1 + seed % 3)


@pytest.mark.parametrize("seed", range(40))
def test_phase1_order2_agrees_with_vertex_enumeration(orc, seed):
    rng = np.random.default_rng(700 + seed)
    K = 10 + 2 * (seed % 2)
    xi, eta = symmetric_ring(rng, K, jitter_of(seed))
    V = orc.vandermonde(2, xi, eta)
    np.testing.assert_allclose(V, textbook_vandermonde9(xi, eta), rtol=1e-15, atol=0)
    st, f, npiv, res = orc.phase1(V, B9)
    verts = vertices(textbook_vandermonde9(xi, eta), B9)
    if not verts:
        assert st != 0
        return
    assert st == 0, "feasible by enumeration but oracle says %d" % st
    assert (f >= 0).all()
    np.testing.assert_allclose(V @ f, B9, atol=1e-10)
    assert np.count_nonzero(f) <= 9
    assert min(np.max(np.abs(f - v)) for v in verts) < 1e-8


def test_vertex_enumeration_cases_cover_both_verdicts(orc):
    # the seeds above must exercise feasible and infeasible neighbourhoods
    verdicts = set()
    for seed in range(40):
        rng = np.random.default_rng(700 + seed)
        K = 10 + 2 * (seed % 2)
        xi, eta = symmetric_ring(rng, K, jitter_of(seed))
        verdicts.add(bool(vertices(textbook_vandermonde9(xi, eta), B9)))
    assert verdicts == {True, False}


@pytest.mark.parametrize("seed", range(20))
def test_point_symmetric_neighbourhood_reduces_to_even_rows(orc, seed):
    # exactly point-symmetric neighbours: averaging a solution with its mirror
    # image keeps every row, so the nine rows are feasible iff some pair
    # weights g_k >= 0 meet the even rows, 2 sum_k g_k (xi^2, xi eta, eta^2)
    # = (2, 0, 2); that 3-row problem is decided by vertex enumeration
    rng = np.random.default_rng(900 + seed)
    xi, eta = symmetric_ring(rng, 10 + 2 * (seed % 2), 0.0)
    half = len(xi) // 2
    even = np.array([xi[:half] ** 2, xi[:half] * eta[:half], eta[:half] ** 2])
    feasible = bool(vertices(even, np.array([1.0, 0.0, 1.0])))
    st, f, _, _ = orc.phase1(orc.vandermonde(2, xi, eta), B9)
    assert (st == 0) == feasible
    if st == 0:
        np.testing.assert_allclose(textbook_vandermonde9(xi, eta) @ f, B9, atol=1e-10)
        assert (f >= 0).all()


def stencil_weights(orc, x, y, h, order, R=2.0):
    n = len(x)
    nb = orc.neighbours(x, y, h, R=R)
    w = orc.solve_weights(x, y, np.ones(n, dtype=np.uint8), nb, h, order)
    return w


def test_cubic_polynomials_reproduced(orc):
    h = 0.05
    x, y, _ = vrm_inputs.random_cloud(1600, h=h, jitter=0.3, seed=21)
    w2 = stencil_weights(orc, x, y, h, 2, R=2.5)
    w1 = stencil_weights(orc, x, y, h, 1, R=2.5)
    ok2 = np.isin(w2["status"], (1, 2))
    edge = np.max(np.abs(x)) - 3 * h
    inner = (np.abs(x) < edge) & (np.abs(y) < edge)
    assert ok2[inner].all()  # away from the cloud's edge every particle has one
    worst1 = 0.0
    for order, w, ok in ((2, w2, ok2), (1, w1, np.isin(w1["status"], (1, 2)))):
        for i in np.nonzero(ok)[0]:
            c = w["cols"][i]
            fv = w["f"][i][c >= 0]
            xi = (x[c[c >= 0]] - x[i]) / h
            eta = (y[c[c >= 0]] - y[i]) / h
            for a, b in MONOMIALS:
                got = np.sum(fv * xi ** a * eta ** b) if (a, b) != (0, 0) else 0.0
                if order == 2 or a + b <= 2:
                    assert abs(got - lap_at_zero(a, b)) < 1e-9, (order, i, a, b, got)
                else:
                    worst1 = max(worst1, abs(got))
    # the cubic rows are what n = 2 adds: n = 1 stencils miss them
    assert worst1 > 1e-2


def laplacian_error(orc, h, order, seed=3):
    x, y, _ = vrm_inputs.gaussian_mixture_cloud(h=h, jitter=0.3, seed=seed, half_width=1.0)
    w = stencil_weights(orc, x, y, h, order, R=2.5)
    u = np.sin(2 * x) * np.cos(3 * y) + x ** 3 * y
    lu = -13.0 * np.sin(2 * x) * np.cos(3 * y) + 6 * x * y
    acc = w["fii"] * u
    for t in range(w["cols"].shape[1]):
        c = w["cols"][:, t]
        acc = acc + np.where(c >= 0, w["f"][:, t] * u[np.maximum(c, 0)], 0.0)
    inner = (np.abs(x) < 0.6) & (np.abs(y) < 0.6)
    ok = np.isin(w["status"], (1, 2))
    assert ok[inner].mean() > 0.999  # R = 2.5: stencils exist almost everywhere
    inner &= ok
    return np.max(np.abs(acc / h ** 2 - lu)[inner])


def test_consistency_order_in_h(orc):
    e2 = [laplacian_error(orc, h, 2) for h in (0.04, 0.02, 0.01)]
    e1 = [laplacian_error(orc, h, 1) for h in (0.04, 0.02, 0.01)]
    for a, b in zip(e2, e2[1:]):
        assert a / b > 3.0  # O(h^2)
    for a, b in zip(e1, e1[1:]):
        assert 1.2 < a / b < 3.0  # O(h)
    assert e2[-1] < 0.1 * e1[-1]


def test_lattice_small_neighbourhood_feasible(orc):
    # on the lattice the four axis neighbours come first (d2 = h^2) and their
    # symmetric stencil meets all nine rows: the small neighbourhood suffices
    h = 1.0 / 32
    x, y = vrm_inputs.lattice(h, -0.5, 0.5)
    w = stencil_weights(orc, x, y, h, 2)
    inner = (np.abs(x) < 0.4) & (np.abs(y) < 0.4)
    assert (w["status"][inner] == 1).all()
    xi = np.array([1.0, 0.0, -1.0, 0.0])
    eta = np.array([0.0, 1.0, 0.0, -1.0])
    np.testing.assert_array_equal(textbook_vandermonde9(xi, eta) @ np.ones(4), B9)


def test_nine_weights_kept(orc):
    h = 0.05
    x, y, _ = vrm_inputs.random_cloud(900, h=h, jitter=0.3, seed=22)
    w = stencil_weights(orc, x, y, h, 2, R=2.5)
    assert w["cols"].shape[1] == orc.stencil_width(2) == 12
    nnz = (w["cols"] >= 0).sum(1)
    assert nnz.max() == 9
    ok = np.isin(w["status"], (1, 2))
    # f~_ii = -sum of the kept weights: nothing was dropped
    np.testing.assert_allclose(w["fii"][ok], -w["f"][ok].sum(1), rtol=1e-14, atol=0)
    assert (w["f"] >= 0).all()


def test_growth_control_bound_h4(orc):
    h = 0.05
    x, y, g = vrm_inputs.random_cloud(900, h=h, jitter=0.3, seed=23, field="random")
    g = g * np.exp(np.random.default_rng(5).uniform(-12, 0, g.size))
    nu, dt = 1e-3, 0.0
    _, _, _, st2 = orc.step(x, y, g, h, nu, dt, order=2, R=2.5)
    _, _, _, st1 = orc.step(x, y, g, h, nu, dt, order=1, R=2.5)
    a = np.abs(g)
    order = sorted(range(len(a)), key=lambda i: (a[i], i))
    total = sum(Fraction(v) for v in a)
    for hp, st in (((h * h * h) * h, st2), (h * h * h, st1)):
        bound = Fraction(hp) * total
        s, k = Fraction(0), 0
        for i in order:
            if s + Fraction(a[i]) > bound:
                break
            s += Fraction(a[i])
            k += 1
        assert st["n_diffused"] == len(a) - k
    assert st2["n_diffused"] > st1["n_diffused"]
