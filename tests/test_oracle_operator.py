"""Pins of the oracle's growth control, operator and time step.

* Sec. 3.5: the left-out set is the longest prefix by (|Gamma|, i) within
  C_diff h^{n+2} ||Gamma||_1, checked with exact rational arithmetic.
* Sec. 3.2 (proof of Thm. consistency): the operator reproduces the
  Laplacian of quadratics exactly at every diffused particle.
* Sec. 3.4: sum dGamma = 0, sum x dGamma = 0 and, for the reduced
  operator, sum |x|^2 dGamma = 4 nu sum_{i in D} Gamma_i.
* Thm. stability: ||Gamma^{n+1}||_1 <= ||Gamma^n||_1 when
  nu dt <= -1/f_ii for all i.
* Sec. 5: single Dirac start (golden file) and second-order convergence of the
  heat-equation Lamb-Oseen run against the closed form.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import vrm_inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def exact_reduce(gamma, c_bound):
    """Longest prefix of (|Gamma|, i) whose exact sum stays within
    c_bound * ||Gamma||_1 (rational arithmetic)."""
    a = [Fraction(abs(float(g))) for g in gamma]
    total = sum(a)
    bound = Fraction(c_bound) * total
    order = sorted(range(len(a)), key=lambda i: (a[i], i))
    d = np.ones(len(a), np.uint8)
    cum = Fraction(0)
    for i in order:
        if cum + a[i] > bound:
            break
        cum += a[i]
        d[i] = 0
    return d


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("c_bound", [1e-3, 0.05, 0.5])
def test_reduce_matches_exact_prefix(orc, seed, c_bound):
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(500) * np.exp(rng.uniform(-20, 0, 500))
    g[::17] = 0.0
    g[5::23] = g[4::23][: len(g[5::23])]  # exact ties in |Gamma|
    d = orc.reduce(g, c_bound)
    np.testing.assert_array_equal(d, exact_reduce(g, c_bound))
    assert not d[g == 0].any()


def test_reduce_edge_cases(orc):
    assert orc.reduce(np.zeros(0), 0.1).size == 0
    assert not orc.reduce(np.zeros(10), 0.1).any()
    g = np.array([1.0, -2.0, 3.0])
    assert orc.reduce(g, 0.0).all()
    assert not orc.reduce(g, 1.0).any()
    # ties: equal |Gamma| leave in index order
    g = np.array([1.0, 1.0, 1.0, 1.0])
    np.testing.assert_array_equal(orc.reduce(g, 0.5), [0, 0, 1, 1])


def operator(orc, x, y, g, h, nu=1.0, c_diff=1.0):
    p = orc.pipeline(x, y, g, h, nu, c_diff=c_diff)
    return p


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_polynomial_exactness(orc, seed):
    # sum_j f_ij (phi(x_j) - phi(x_i)) = Delta phi(x_i) for quadratic phi
    h = 0.05
    x, y, g = vrm_inputs.random_cloud(1200, h=h, jitter=0.35, seed=seed)
    p = operator(orc, x, y, g, h)
    X, Y, w = p["x"], p["y"], p["w"]
    rng = np.random.default_rng(seed)
    a, b, c, d, e = rng.standard_normal(5)
    phi = lambda u, v: a * u * u + b * u * v + c * v * v + d * u + e * v
    lap = 2 * a + 2 * c
    ok = np.nonzero((w["status"] == 1) | (w["status"] == 2))[0]
    assert len(ok) > 100
    for i in ok:
        js = w["cols"][i][w["cols"][i] >= 0]
        fs = w["f"][i][: len(js)]
        val = np.sum(fs * (phi(X[js], Y[js]) - phi(X[i], Y[i]))) / (h * h)
        assert abs(val - lap) < 1e-9 * (1 + abs(lap))
        assert w["fii"][i] <= 0
        assert abs(w["fii"][i] + fs.sum()) < 1e-13 * fs.sum()


@pytest.mark.parametrize("seed", [0, 1])
def test_conservation_of_reduced_operator(orc, seed):
    h, nu = 0.05, 0.7
    x, y, g = vrm_inputs.random_cloud(1500, h=h, jitter=0.3, seed=seed)
    p = operator(orc, x, y, g, h, nu=nu, c_diff=5.0)
    X, Y, dg = p["x"], p["y"], p["dgamma"]
    D = p["diffused"][: len(g)].astype(bool)
    assert 0 < D.sum() < len(g)
    scale = nu / h ** 2 * 16 * np.abs(g).sum()
    assert abs(dg.sum()) < 1e-13 * scale
    assert abs(np.sum(X * dg)) < 1e-13 * scale
    assert abs(np.sum(Y * dg)) < 1e-13 * scale
    i2 = np.sum((X * X + Y * Y) * dg)
    assert abs(i2 - 4 * nu * g[D].sum()) < 1e-11 * (abs(4 * nu * np.abs(g).sum()))


def test_stability_l1_nonincreasing(orc):
    h, nu = 0.05, 1.0
    x, y, g = vrm_inputs.random_cloud(900, h=h, jitter=0.3, seed=4, field="noise")
    p = operator(orc, x, y, g, h, nu=nu)
    fmax = -p["w"]["fii"].min()
    dt = h * h / (nu * fmax)  # nu dt (-f_ii)/h^2 <= 1 for all i
    x2, y2, g2, st = orc.step(x, y, g, h, nu, dt)
    assert st["max_dt_ratio"] <= 1 + 1e-12
    assert np.abs(g2).sum() <= np.abs(g).sum() * (1 + 1e-13)
    assert abs(g2.sum() - g.sum()) < 1e-13 * np.abs(g).sum()
    # twice the bound breaks it (Thm. stability, converse)
    x3, y3, g3, st = orc.step(x, y, g, h, nu, 4 * dt)
    assert np.abs(g3).sum() > np.abs(g).sum()


def test_single_dirac_golden(orc):
    # Sec. 5: the Lamb-Oseen run starts from one Dirac; see golden file
    gold = json.load(open(os.path.join(GOLDEN, "single_particle.json")))
    h, nu, G = gold["h"], gold["nu"], gold["gamma"]
    p = operator(orc, np.array([0.0]), np.array([0.0]), np.array([G]), h, nu=nu)
    assert len(p["x"]) == 9
    for s in range(8):
        assert abs(p["x"][1 + s] - gold["inserted"][s][0]) < 1e-15
        assert abs(p["y"][1 + s] - gold["inserted"][s][1]) < 1e-15
    assert abs(-p["w"]["fii"][0] - gold["sum_f_scaled"]) < 1e-14
    assert abs(p["dgamma"][0] - gold["dgamma0"]) < 1e-13 * abs(gold["dgamma0"])
    assert abs(p["dgamma"].sum()) < 1e-14


def weak_error(x, y, g, gamma, nu, t, centres, sigma):
    """max_k |sum_i Gamma_i phi_k(x_i) - int omega(t) phi_k| / Gamma for
    Gaussian test functions phi_k = exp(-|x-c_k|^2/(2 sigma^2)); the exact
    integral of the Lamb-Oseen field against phi_k is
    Gamma sigma^2/(2 nu t + sigma^2) exp(-|c_k|^2/(2 (2 nu t + sigma^2)))."""
    err = 0.0
    s2 = 2 * nu * t + sigma ** 2
    for cx, cy in centres:
        num = np.sum(g * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * sigma ** 2)))
        ex = gamma * sigma ** 2 / s2 * math.exp(-(cx * cx + cy * cy) / (2 * s2))
        err = max(err, abs(num - ex) / gamma)
    return err


def test_lamb_oseen_heat_convergence(orc):
    # Heat-equation Lamb-Oseen run with Euler and dt = (1/8)(r h)^2/(4 nu)
    # (Sec. 5.1) on lattices with binary-exact coordinates (h = 2^-k), so that
    # the particle locations are symmetric as in the paper's second-order
    # observation (Sec. 5.1); the weak error against the closed form falls
    # like h^2.
    gamma, nu, t0, t1 = 1.0, 1e-3, 1.0, 1.125
    centres = [(0.0, 0.0), (0.03, 0.0), (0.05, 0.04), (-0.08, 0.02), (0.0, -0.1)]
    errs = []
    hs = [1 / 32, 1 / 64, 1 / 128]
    for h in hs:
        x, y, g = vrm_inputs.lamb_oseen_lattice(h, gamma, nu, t0, eps=1e-8)
        dt = (0.5 * h) ** 2 / (4 * nu) / 8
        steps = int(round((t1 - t0) / dt))
        dt = (t1 - t0) / steps
        g0 = g.sum()
        for _ in range(steps):
            x, y, g, st = orc.step(x, y, g, h, nu, dt)
            assert st["no_stencil"] == 0
        # circulation is conserved to round-off by the heat-equation steps
        assert abs(g.sum() - g0) < 1e-12 * gamma
        errs.append(weak_error(x, y, g, gamma, nu, t1, centres, 0.03))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]
    assert min(rates) > 1.8, (errs, rates)
