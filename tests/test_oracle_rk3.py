"""Pins of the oracle's SSP-RK3 step with Lamb-Oseen advection: the velocity
against the closed form in polar form, third-order time accuracy on the pure
advection of a point (exact circular orbit), the step without velocity
against three operator applications, and conservation."""
import math

import numpy as np

import vrm_inputs


def test_velocity_closed_form(orc):
    gamma, nu, t = 1.3, 1e-3, 1.7
    r = np.array([1e-4, 0.01, 0.05, 0.1, 0.3])
    th = np.array([0.1, 1.0, 2.0, 3.0, 5.0])
    x, y = r * np.cos(th), r * np.sin(th)
    u, v = orc.lamb_oseen_velocity(x, y, gamma, nu, t)
    ut = gamma / (2 * math.pi * r) * -np.expm1(-r * r / (4 * nu * t))  # 1 - exp(-a), accurate at small a
    assert np.allclose(u, -np.sin(th) * ut, rtol=1e-13, atol=0)
    assert np.allclose(v, np.cos(th) * ut, rtol=1e-13, atol=0)
    # radial component zero; the centre does not move
    assert np.max(np.abs(u * x + v * y)) < 1e-15
    u0, v0 = orc.lamb_oseen_velocity(np.array([0.0]), np.array([0.0]), gamma, nu, t)
    assert u0[0] == 0.0 and v0[0] == 0.0


def test_rk3_orbit_is_third_order(orc):
    # far from the core (r^2 >> 4 nu t) the field is the point vortex u = Gamma/(2 pi r):
    # one particle (zero circulation, nothing diffuses) orbits at angular
    # speed Gamma/(2 pi r^2); the RK3 position error after a fixed time
    # falls like dt^3
    gamma, nu, t0, r0, T = 1.0, 1e-6, 1.0, 0.5, 0.5
    omega = gamma / (2 * math.pi * r0 * r0)
    errs = []
    for steps in (10, 20, 40):
        dt = T / steps
        x, y, g = np.array([r0]), np.array([0.0]), np.array([0.0])
        t = t0
        for _ in range(steps):
            x, y, g, _ = orc.rk3_step(x, y, g, 0.05, nu, t, dt, vel=dict(gamma=gamma, nu=nu))
            t += dt
        errs.append(math.hypot(x[0] - r0 * math.cos(omega * T), y[0] - r0 * math.sin(omega * T)))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(rates) > 2.8, (errs, rates)


def test_rk3_without_velocity_is_three_operator_applications(orc):
    x, y, g = vrm_inputs.random_cloud(400, h=0.05, jitter=0.3, seed=4)
    h, nu, dt = 0.05, 1e-3, 0.05
    X, Y, G, st = orc.rk3_step(x, y, g, h, nu, 1.0, dt)
    # positions are the inserted cloud, unmoved
    p = orc.pipeline(x, y, g, h, nu)
    assert np.array_equal(X, p["x"]) and np.array_equal(Y, p["y"])
    # with fixed positions the stages reduce to G3 = G0 + dt L G0 + dt^2/2 L^2 G0 + dt^3/6 L^3 G0
    n2 = len(X)
    G0 = np.zeros(n2)
    G0[:len(g)] = g
    L = lambda v: orc.apply(n2, v, p["diffused"], p["w"], p["const"]["nu_over_h2"])
    L1 = L(G0)
    L2 = L(L1)
    L3 = L(L2)
    ref = G0 + dt * L1 + dt ** 2 / 2 * L2 + dt ** 3 / 6 * L3
    assert np.max(np.abs(G - ref)) <= 1e-13 * np.max(np.abs(g))
    # circulation conserved to round-off
    assert abs(G.sum() - g.sum()) <= 1e-13 * np.abs(g).sum()


def test_rk3_lamb_oseen_conserves_and_tracks_the_closed_form(orc):
    h, gamma, nu, t0 = 1 / 32, 1.0, 1e-3, 1.0
    x, y, g = vrm_inputs.lamb_oseen_lattice(h, gamma, nu, t0, eps=1e-8)
    # dt within the diffusive bound (r h)^2/(4 nu) and an advective CFL of
    # 1/4 (peak azimuthal speed about 1.43 at r = 2.24 sqrt(nu t))
    dt = min((0.5 * h) ** 2 / (4 * nu), 0.25 * h / 1.43)
    t = t0
    g0 = g.sum()
    for _ in range(4):
        x, y, g, st = orc.rk3_step(x, y, g, h, nu, t, dt, vel=dict(gamma=gamma, nu=nu))
        t += dt
        # insertion runs on the step's initial cloud only: the shear of the
        # later stages leaves a few particles without a stencil (they do not
        # diffuse in that stage; conservation holds)
        assert st["no_stencil"] <= 0.01 * 3 * st["n_diffused"]
    assert abs(g.sum() - g0) < 1e-12
    # the vortex stays centred (the discrete advection moves the first
    # moments only at the level of the lattice's asymmetry)
    assert abs(np.sum(g * x)) < 1e-6 and abs(np.sum(g * y)) < 1e-6
    # second moment: d/dt sum Gamma |x|^2 = 4 nu sum Gamma for the heat part;
    # rotation leaves |x| unchanged
    I2 = np.sum(g * (x * x + y * y))
    I2_0 = 4 * nu * t0 * g0  # closed form of the Lamb-Oseen second moment
    assert abs(I2 - 4 * nu * t * g0) < 0.05 * (I2 - I2_0 + 1e-30) + 1e-6


def test_rk3_two_point_vortices_corotate(orc):
    # self-induced velocity (direct sum): two equal vortices d apart (d >> eps,
    # no neighbours, growth-control bound >= 1 so nothing diffuses) turn about
    # their midpoint at Gamma_total / (2 pi d^2); RK3 keeps the distance
    gamma, d, eps = 1.0, 5.0, 0.1
    x, y, g = np.array([-d / 2, d / 2]), np.array([0.0, 0.0]), np.array([gamma, gamma])
    om = 2 * gamma / (2 * math.pi * d * d)
    T = 0.5 / om
    steps = 40
    dt = T / steps
    t = 1.0
    for _ in range(steps):
        x, y, g, st = orc.rk3_step(x, y, g, 1.0, 1e-3, t, dt, vel=dict(eps=eps))
        t += dt
    assert len(x) == 2 and st["n_diffused"] == 0
    ang = om * T
    assert abs(x[1] - d / 2 * math.cos(ang)) < 1e-5 and abs(y[1] - d / 2 * math.sin(ang)) < 1e-5
    assert abs(math.hypot(x[1] - x[0], y[1] - y[0]) - d) < 1e-5
