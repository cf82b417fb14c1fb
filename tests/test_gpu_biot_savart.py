"""The direct-sum smoothed Biot-Savart velocity on the GPU (vrm_biot_savart)
against the oracle's FP64 direct sum, the Lamb-Oseen velocity it recovers
from a particle sample, and the RK3 step with the particles' own velocity.

Tolerance: the pair terms are fp32 on hi/lo-split positions with fp32 tile
sums, so a velocity is within a few 1e-7 (bound used: 2e-6) of
S_t = sum_j |Gamma_j| |K_eps(x_t - x_j)| of its exact value."""
import math

import numpy as np
import pytest

import vrm_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1508_06379_gb300 as v
    v.build()
    return v


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def kernel_scale(xs, ys, g, xt, yt, eps):
    dx = xt[:, None] - xs[None, :]
    dy = yt[:, None] - ys[None, :]
    r2 = dx * dx + dy * dy
    with np.errstate(divide="ignore", invalid="ignore"):
        k = np.where(r2 > 0, -np.expm1(-r2 / eps ** 2) / (2 * math.pi * np.sqrt(r2)), 0.0)
    return k @ np.abs(g)


def test_direct_sum_matches_oracle(lib, orc):
    rng = np.random.default_rng(41)
    n, m, eps = 3000, 2000, 0.03
    xs, ys = rng.uniform(-0.7, 1.3, n), rng.uniform(-1.0, 1.0, n)
    g = rng.normal(0.0, 1.0, n) * 1e-3
    xt = np.concatenate([xs[:500], rng.uniform(-0.8, 1.4, m - 500)])  # some targets on sources
    yt = np.concatenate([ys[:500], rng.uniform(-1.1, 1.1, m - 500)])
    ctx = lib.VRM(h=eps / 3, nu=1e-3)
    u, v = ctx.biot_savart(cu(xs), cu(ys), cu(g), n, cu(xt), cu(yt), m, eps)
    uo, vo = orc.biot_savart(xs, ys, g, xt, yt, eps)
    S = kernel_scale(xs, ys, g, xt, yt, eps)
    err = np.maximum(np.abs(u.cpu().numpy() - uo), np.abs(v.cpu().numpy() - vo))
    assert np.all(err <= 2e-6 * S + 1e-300), float(np.max(err / S))


def test_lamb_oseen_velocity_from_particles(lib, orc):
    gamma, nu, t0, h = 1.0, 1e-3, 1.0, 0.005
    x, y, g = vrm_inputs.lamb_oseen_lattice(h, gamma, nu, t0, eps=1e-10)
    gx = np.linspace(-0.3, 0.3, 61)
    XT, YT = np.meshgrid(gx, gx)
    xt, yt = XT.ravel(), YT.ravel()
    ctx = lib.VRM(h=h, nu=nu)
    u, v = ctx.biot_savart(cu(x), cu(y), cu(g), len(x), cu(xt), cu(yt), len(xt), 3 * h)
    u, v = u.cpu().numpy(), v.cpu().numpy()
    ue, ve = orc.lamb_oseen_velocity(xt, yt, gamma, nu, t0)
    e_gpu = math.sqrt(np.sum((u - ue) ** 2 + (v - ve) ** 2) / np.sum(ue ** 2 + ve ** 2))
    uo, vo = orc.biot_savart(x, y, g, xt, yt, 3 * h)
    e_orc = math.sqrt(np.sum((uo - ue) ** 2 + (vo - ve) ** 2) / np.sum(ue ** 2 + ve ** 2))
    assert abs(e_gpu - e_orc) <= 1e-5 * max(e_orc, 1e-3) + 1e-7 and e_gpu < 0.02


def test_rk3_with_self_induced_velocity(lib, orc):
    # a Lamb-Oseen sample moving with its own smoothed velocity (eps = 3h):
    # positions follow the oracle's step within the fp32 velocity error,
    # circulation is conserved and the vortex stays centred
    gamma, nu, t0, h = 1.0, 1e-3, 1.0, 0.02
    x, y, g = vrm_inputs.lamb_oseen_lattice(h, gamma, nu, t0, eps=1e-10)
    dt = 0.25 * h / 1.43
    n = len(x)
    cap = 4 * n + 1024
    xb = torch.zeros(cap, dtype=torch.float64, device="cuda")
    yb = torch.zeros(cap, dtype=torch.float64, device="cuda")
    xb[:n] = cu(x)
    yb[:n] = cu(y)
    go = torch.zeros(cap, dtype=torch.float64, device="cuda")
    ctx = lib.VRM(h=h, nu=nu)
    n2, st = ctx.rk3_step(xb, yb, n, cu(g), go, t0, dt, dict(eps=3 * h))
    X, Y, G = xb[:n2].cpu().numpy(), yb[:n2].cpu().numpy(), go[:n2].cpu().numpy()
    Xo, Yo, Go, sto = orc.rk3_step(x, y, g, h, nu, t0, dt, vel=dict(eps=3 * h))
    assert n2 == len(Xo)
    umax = 1.5
    assert np.max(np.abs(X - Xo)) <= 1e-5 * umax * dt and np.max(np.abs(Y - Yo)) <= 1e-5 * umax * dt
    assert abs(G.sum() - g.sum()) < 1e-13
    assert abs(np.sum(G * X)) < 1e-6 and abs(np.sum(G * Y)) < 1e-6
    # circulations agree to the scale of the diffusion increment where the stencils agree
    scale = dt * nu / h ** 2 * np.abs(g).max() * 16
    assert np.median(np.abs(G - Go)) <= 1e-9 * scale + 1e-15
