"""Pins of the oracle's smoothed Biot-Savart velocity (Sec. 5, Eq.
smoothkernel): the closed form of one blob, the point-vortex far field,
superposition and antisymmetry, zero self-induced velocity, and the
Lamb-Oseen velocity recovered from a particle sample (L2 error falling with
h, the smoothing error O(eps^2))."""
import math

import numpy as np

import vrm_inputs


def test_single_blob_closed_form(orc):
    eps = 0.03
    r = np.array([1e-6, 0.005, 0.03, 0.1, 1.0])
    th = 0.7
    u, v = orc.biot_savart([0.0], [0.0], [1.7], r * math.cos(th), r * math.sin(th), eps)
    ut = 1.7 * -np.expm1(-(r / eps) ** 2) / (2 * math.pi * r)
    assert np.allclose(u, -math.sin(th) * ut, rtol=1e-12, atol=1e-300)
    assert np.allclose(v, math.cos(th) * ut, rtol=1e-12, atol=1e-300)
    # far field: the point vortex Gamma/(2 pi r)
    assert abs(ut[-1] - 1.7 / (2 * math.pi)) < 1e-15
    # at the source itself the velocity is zero
    u0, v0 = orc.biot_savart([0.2], [-0.1], [1.7], [0.2], [-0.1], eps)
    assert u0[0] == 0.0 and v0[0] == 0.0


def test_superposition_and_pair_symmetry(orc):
    rng = np.random.default_rng(5)
    xs, ys, g = rng.uniform(-1, 1, 50), rng.uniform(-1, 1, 50), rng.normal(0, 1, 50)
    xt, yt = rng.uniform(-1, 1, 30), rng.uniform(-1, 1, 30)
    u, v = orc.biot_savart(xs, ys, g, xt, yt, 0.1)
    u1, v1 = orc.biot_savart(xs[:20], ys[:20], g[:20], xt, yt, 0.1)
    u2, v2 = orc.biot_savart(xs[20:], ys[20:], g[20:], xt, yt, 0.1)
    assert np.allclose(u, u1 + u2, rtol=0, atol=1e-13) and np.allclose(v, v1 + v2, rtol=0, atol=1e-13)
    # the self-induced velocities of a cloud carry no net impulse change:
    # sum_i Gamma_i u(x_i) = 0 (the kernel is odd)
    us, vs = orc.biot_savart(xs, ys, g, xs, ys, 0.1)
    assert abs(np.sum(g * us)) < 1e-12 and abs(np.sum(g * vs)) < 1e-12


def test_lamb_oseen_velocity_from_particles(orc):
    # particles sampling omega(t0) on lattices: the smoothed velocity with
    # eps = 3h approaches the analytic Lamb-Oseen velocity as h falls
    gamma, nu, t0 = 1.0, 1e-3, 1.0
    gx = np.linspace(-0.3, 0.3, 41)
    XT, YT = np.meshgrid(gx, gx)
    xt, yt = XT.ravel(), YT.ravel()
    ue, ve = orc.lamb_oseen_velocity(xt, yt, gamma, nu, t0)
    errs = []
    for h in (0.02, 0.01, 0.005):
        x, y, g = vrm_inputs.lamb_oseen_lattice(h, gamma, nu, t0, eps=1e-10)
        u, v = orc.biot_savart(x, y, g, xt, yt, 3 * h)
        errs.append(math.sqrt(np.sum((u - ue) ** 2 + (v - ve) ** 2) / np.sum(ue ** 2 + ve ** 2)))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.02, errs
