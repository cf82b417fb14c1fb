"""Seeded synthetic particle clouds for the VRM diffusion operator.

This module only draws inputs: positions and circulations sampled from
closed-form vorticity fields.  It holds none of the redistribution method's
arithmetic and is shared by the tests, the benchmark and the oracle checks.

Workloads (the paper has no dataset; every cloud here is synthetic):

* ``lamb_oseen_lattice``: the Lamb-Oseen vortex of Sec. 5,
  omega(t, x) = Gamma/(4 pi nu t) exp(-|x|^2/(4 nu t)), sampled on a uniform
  lattice k h - 1 (k = 0..2/h) with Gamma_i = omega(t0, x_i) h^2 (midpoint
  quadrature), optionally keeping |omega| > eps only.
* ``gaussian_mixture_cloud``: a jittered lattice carrying a sum of Gaussian
  vortices, omega = sum_k Gamma_k/(2 pi s_k^2) exp(-|x-c_k|^2/(2 s_k^2)).
* ``batched_clouds``: many independent mixture clouds of log-uniform size.
* ``mlp_params``, ``mlp_rows``, ``mlp_vector``: random parameters, input rows
  and vectors for the weight-proposal network (rows of exactly
  bf16-representable values: multiples of 1/64 in [-2, 2] and 0/1 masks).
"""
import math

import numpy as np

SEED_BASE = 1508000


def lamb_oseen_omega(x, y, gamma=1.0, nu=1e-3, t=1.0):
    r2 = x * x + y * y
    return gamma / (4.0 * math.pi * nu * t) * np.exp(-r2 / (4.0 * nu * t))


def lamb_oseen_velocity(x, y, gamma=1.0, nu=1e-3, t=1.0):
    """Azimuthal velocity of the Lamb-Oseen vortex (Sec. 5)."""
    r2 = x * x + y * y
    with np.errstate(invalid="ignore", divide="ignore"):
        s = gamma / (2.0 * math.pi * r2) * (1.0 - np.exp(-r2 / (4.0 * nu * t)))
    s = np.where(r2 > 0, s, 0.0)
    return -y * s, x * s


def lattice(h, lo=-1.0, hi=1.0):
    n = int(round((hi - lo) / h)) + 1
    k = np.arange(n, dtype=np.float64)
    c = k * h + lo
    X, Y = np.meshgrid(c, c, indexing="xy")
    return X.ravel().copy(), Y.ravel().copy()


def lamb_oseen_lattice(h=0.02, gamma=1.0, nu=1e-3, t0=1.0, eps=1e-10, lo=-1.0, hi=1.0):
    """Lattice sample of the Lamb-Oseen vortex; eps=None keeps every point."""
    x, y = lattice(h, lo, hi)
    w = lamb_oseen_omega(x, y, gamma, nu, t0)
    if eps is not None:
        keep = np.abs(w) > eps
        x, y, w = x[keep], y[keep], w[keep]
    return x, y, w * h * h


def _mixture(rng, n_modes, centre_box, sigma_lo, sigma_hi):
    c = rng.uniform(-centre_box, centre_box, size=(n_modes, 2))
    g = rng.standard_normal(n_modes)
    s = rng.uniform(sigma_lo, sigma_hi, size=n_modes)
    return c, g, s


def mixture_omega(x, y, centres, gammas, sigmas):
    w = np.zeros_like(x)
    for (cx, cy), g, s in zip(centres, gammas, sigmas):
        r2 = (x - cx) ** 2 + (y - cy) ** 2
        w += g / (2.0 * math.pi * s * s) * np.exp(-r2 / (2.0 * s * s))
    return w


def gaussian_mixture_cloud(h=2e-3, side=None, jitter=0.3, seed=SEED_BASE + 2, n_modes=8, half_width=1.0):
    """Jittered lattice on [-half_width, half_width]^2 with spacing h, uniform
    jitter U(-jitter h, jitter h) per coordinate, carrying a mixture of
    n_modes Gaussians (centres U[-0.8 w, 0.8 w]^2, Gamma_k ~ N(0,1),
    sigma_k ~ U[0.05 w, 0.15 w], w = half_width)."""
    rng = np.random.default_rng(seed)
    if side is None:
        side = int(round(2.0 * half_width / h)) + 1
    k = np.arange(side, dtype=np.float64)
    c = k * h - half_width
    X, Y = np.meshgrid(c, c, indexing="xy")
    x = X.ravel() + rng.uniform(-jitter * h, jitter * h, size=X.size)
    y = Y.ravel() + rng.uniform(-jitter * h, jitter * h, size=Y.size)
    cen, g, s = _mixture(rng, n_modes, 0.8 * half_width, 0.05 * half_width, 0.15 * half_width)
    w = mixture_omega(x, y, cen, g, s)
    return x, y, w * h * h


def batched_clouds(n_clouds=64, n_lo=1e4, n_hi=5e5, h_lo=1e-3, h_hi=4e-3, seed=SEED_BASE + 3, jitter=0.3):
    """Independent mixture clouds of log-uniform size N_c in [n_lo, n_hi] and
    spacing h_c ~ U[h_lo, h_hi]; cloud c is a sqrt(N_c)-sided jittered lattice
    of half width L/2 = sqrt(N_c) h_c / 2 carrying the mixture scaled to it.
    Returns a list of (x, y, gamma, h)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_clouds):
        nc = int(math.floor(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        hc = float(rng.uniform(h_lo, h_hi))
        side = max(2, int(round(math.sqrt(nc))))
        half = 0.5 * side * hc
        sub_seed = int(rng.integers(0, 2**31 - 1))
        x, y, g = gaussian_mixture_cloud(h=hc, side=side, jitter=jitter, seed=sub_seed, half_width=half)
        out.append((x, y, g, hc))
    return out


def random_cloud(n, h=0.1, jitter=0.3, seed=0, field="mixture"):
    """Small jittered lattice with about n points (tests)."""
    side = max(2, int(round(math.sqrt(n))))
    half = 0.5 * (side - 1) * h
    rng = np.random.default_rng(seed)
    k = np.arange(side, dtype=np.float64)
    c = k * h - half
    X, Y = np.meshgrid(c, c, indexing="xy")
    x = X.ravel() + rng.uniform(-jitter * h, jitter * h, size=X.size)
    y = Y.ravel() + rng.uniform(-jitter * h, jitter * h, size=Y.size)
    if field == "mixture":
        cen, g, s = _mixture(rng, 4, 0.6 * max(half, h), 0.15 * max(half, h), 0.4 * max(half, h))
        w = mixture_omega(x, y, cen, g, s)
    else:
        w = rng.standard_normal(x.size)
    return x, y, w * h * h


def uniform_scatter(n, half_width=1.0, seed=0):
    """Uniformly scattered points with standard normal circulations (tests)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-half_width, half_width, n)
    y = rng.uniform(-half_width, half_width, n)
    g = rng.standard_normal(n)
    return x, y, g


MLP_SHAPES = ((256, 96), (256, 256), (256, 256), (32, 256))


def mlp_params(seed=SEED_BASE + 4, bias_scale=0.05):
    """Flat parameter vector [W1, b1, ..., W4, b4]: W ~ N(0, 1/fan_in), b ~ N(0, bias_scale^2)."""
    rng = np.random.default_rng(seed)
    parts = []
    for out, inp in MLP_SHAPES:
        parts.append(rng.normal(0.0, 1.0 / math.sqrt(inp), out * inp))
        parts.append(rng.normal(0.0, bias_scale, out))
    return np.concatenate(parts)


def mlp_rows(rows, seed=SEED_BASE + 5):
    """Network input rows [rows, 128]: per row a random number k of filled
    slots (8..32), offsets on the 1/64 grid in [-2, 2], mask 1 on the first k
    slots, zeros elsewhere; and targets [rows, 32]: on filled slots a smooth
    non-negative function of the slot's own offsets, max(xi_x, 0)/2 +
    xi_y^2/8, zero elsewhere (learnable, unlike noise)."""
    rng = np.random.default_rng(seed)
    X = np.zeros((rows, 128))
    T = np.zeros((rows, 32))
    for r in range(rows):
        k = int(rng.integers(8, 33))
        X[r, :k] = rng.integers(-128, 129, k) / 64.0
        X[r, 32:32 + k] = rng.integers(-128, 129, k) / 64.0
        X[r, 64:64 + k] = 1.0
        T[r, :k] = np.maximum(X[r, :k], 0.0) / 2 + X[r, 32:32 + k] ** 2 / 8
    return X, T


def mlp_vector(seed, n=164640, scale=1.0):
    """A random vector of the parameter length (e.g. a gradient)."""
    return np.random.default_rng(seed).normal(0.0, scale, n)

