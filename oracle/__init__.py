"""CPU oracle of the VRM diffusion operator (arXiv 1508.06379).

TEST INFRASTRUCTURE ONLY: a plain FP64 C restatement of the method
(``vrm_oracle.c``) with a ctypes wrapper.  Only the tests, the smoke check
and bench.py's CPU-baseline leg import this package; the CUDA library and
its Python binding never do.  ``build()`` compiles the shared object with gcc
(OpenMP, no floating-point contraction).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vrm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile liboracle.so next to the source (gcc, -ffp-contract=off)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Stats(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_long), ("n_out", ctypes.c_long), ("n_diffused", ctypes.c_long),
                ("n_inserted", ctypes.c_long), ("open_segments", ctypes.c_long),
                ("small_ok", ctypes.c_long), ("full_ok", ctypes.c_long), ("no_stencil", ctypes.c_long),
                ("max_pivots", ctypes.c_long), ("rounds", ctypes.c_int), ("max_dt_ratio", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        L.orc_reduce.restype = ctypes.c_long
        L.orc_reduce.argtypes = [P, ctypes.c_long, ctypes.c_double, P]
        L.orc_segment.restype = ctypes.c_int
        L.orc_segment.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_neighbours.restype = ctypes.c_long
        L.orc_neighbours.argtypes = [P, P, ctypes.c_long, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, P, P, ctypes.c_int, P, P]
        L.orc_insertion_offsets.restype = None
        L.orc_insertion_offsets.argtypes = [ctypes.c_double, P, P]
        L.orc_insert.restype = ctypes.c_long
        L.orc_insert.argtypes = [P, P, ctypes.c_long, ctypes.c_long, P, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int, P, P]
        L.orc_close.restype = ctypes.c_long
        L.orc_close.argtypes = [P, P, P, ctypes.c_long, ctypes.c_double, ctypes.c_double, P]
        L.orc_remove_weights.restype = None
        L.orc_remove_weights.argtypes = [P, P, ctypes.c_long, P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, P, P, P]
        L.orc_remove.restype = ctypes.c_long
        L.orc_remove.argtypes = [P, P, P, ctypes.c_long, ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P, P,
                                 P, P]
        L.orc_rows.restype = ctypes.c_int
        L.orc_rows.argtypes = [ctypes.c_int]
        L.orc_stencil_width.restype = ctypes.c_int
        L.orc_stencil_width.argtypes = [ctypes.c_int]
        L.orc_vandermonde_column.restype = None
        L.orc_vandermonde_column.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, P]
        L.orc_phase1.restype = ctypes.c_int
        L.orc_phase1.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P, P]
        L.orc_solve_weights.restype = None
        L.orc_solve_weights.argtypes = [P, P, ctypes.c_long, P, P, P, ctypes.c_int, P, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, P, P]
        L.orc_apply.restype = None
        L.orc_apply.argtypes = [ctypes.c_long, ctypes.c_long, P, P, P, P, P, ctypes.c_int, ctypes.c_double, P]
        L.orc_euler.restype = None
        L.orc_euler.argtypes = [ctypes.c_long, ctypes.c_long, P, P, ctypes.c_double, P]
        L.orc_step.restype = ctypes.c_long
        L.orc_step.argtypes = [P, P, ctypes.c_long, ctypes.c_long, P, P, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                               ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.restype = None
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads():
    return lib().orc_num_threads()


def set_num_threads(t):
    lib().orc_set_num_threads(int(t))


# Derived constants, computed exactly as the oracle's step does.
def constants(h, r=0.5, R=2.0, nu=1.0, c_diff=1.0, order=1):
    rh, Rh = r * h, R * h
    hp = h * h * h
    if order == 2:
        hp = hp * h
    return dict(lo2=rh * rh, hi2=Rh * Rh, Rh=Rh, c_bound=c_diff * hp, nu_over_h2=nu / (h * h))


def reduce(gamma, c_bound):
    """Diffused flags (Sec. 3.5, Eq. reduced_bound): returns uint8[n]."""
    g = _f64(gamma)
    out = np.zeros(len(g), dtype=np.uint8)
    lib().orc_reduce(_p(g), len(g), float(c_bound), _p(out))
    return out


def segment(dx, dy):
    return lib().orc_segment(float(dx), float(dy))


def neighbours(x, y, h, r=0.5, R=2.0, k_cap=32, fp32=False):
    """Annulus neighbourhoods (Eq. neighbourhood), segment masks, small nbhd."""
    x, y = _f64(x), _f64(y)
    n = len(x)
    c = constants(h, r, R)
    count = np.zeros(n, dtype=np.int32)
    idx = np.full((max(n, 1), k_cap), -1, dtype=np.int32)
    mask = np.zeros(n, dtype=np.uint8)
    small = np.full((max(n, 1), 8), -1, dtype=np.int32)
    mx = lib().orc_neighbours(_p(x), _p(y), n, c["lo2"], c["hi2"], c["Rh"], int(bool(fp32)), _p(count), _p(idx),
                              k_cap, _p(mask), _p(small))
    return dict(count=count, idx=idx[:n], mask=mask, small=small[:n], max_count=int(mx))


def insertion_offsets(h):
    ox = np.zeros(8)
    oy = np.zeros(8)
    lib().orc_insertion_offsets(float(h), _p(ox), _p(oy))
    return ox, oy


def insert(x, y, diffused, h, r=0.5, R=2.0, max_rounds=8, capacity=None):
    """Insertion rounds (Sec. 4.2).  Returns (x', y', rounds, open_segments)."""
    n = len(x)
    cap = capacity if capacity is not None else n + 8 * int(np.sum(diffused)) * (max_rounds + 1) + 16
    xb = np.zeros(cap)
    yb = np.zeros(cap)
    xb[:n] = x
    yb[:n] = y
    d = np.ascontiguousarray(diffused, dtype=np.uint8)
    c = constants(h, r, R)
    rounds = ctypes.c_int(0)
    open_ = ctypes.c_long(0)
    n2 = lib().orc_insert(_p(xb), _p(yb), n, cap, _p(d), float(h), c["lo2"], c["hi2"], c["Rh"], int(max_rounds),
                          ctypes.byref(rounds), ctypes.byref(open_))
    if n2 < 0:
        raise ValueError("capacity too small: need %d" % (-n2))
    return xb[:n2].copy(), yb[:n2].copy(), rounds.value, open_.value


def vandermonde(order, xi, eta):
    m = lib().orc_rows(order)
    K = len(xi)
    V = np.zeros((m, K))
    col = np.zeros(9)
    for j in range(K):
        lib().orc_vandermonde_column(order, float(xi[j]), float(eta[j]), _p(col))
        V[:, j] = col[:m]
    return V


def phase1(V, b):
    """Phase-I simplex on V f = b, f >= 0 (Sec. 4.1).  Returns (status, f, pivots, residual)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    b = _f64(b)
    m, K = V.shape
    f = np.zeros(max(K, 1))
    npiv = ctypes.c_int(0)
    res = ctypes.c_double(0)
    st = lib().orc_phase1(m, K, _p(V), _p(b), _p(f), ctypes.byref(npiv), ctypes.byref(res))
    return st, f[:K], npiv.value, res.value


def stencil_width(order):
    """Slots per stencil: at most m nonzero weights (m = 5 for n = 1, 9 for n = 2)."""
    return lib().orc_stencil_width(int(order))


def solve_weights(x, y, diffused, nb, h, order=1, fallback=True, W=None):
    W = stencil_width(order) if W is None else W
    x, y = _f64(x), _f64(y)
    n = len(x)
    k_cap = nb["idx"].shape[1]
    cols = np.full((max(n, 1), W), -1, dtype=np.int32)
    f = np.zeros((max(n, 1), W))
    fii = np.zeros(max(n, 1))
    status = np.zeros(max(n, 1), dtype=np.uint8)
    npiv = np.zeros(max(n, 1), dtype=np.int32)
    d = np.ascontiguousarray(diffused, dtype=np.uint8)
    cnt = np.ascontiguousarray(nb["count"], dtype=np.int32)
    idx = np.ascontiguousarray(nb["idx"], dtype=np.int32)
    small = np.ascontiguousarray(nb["small"], dtype=np.int32)
    lib().orc_solve_weights(_p(x), _p(y), n, _p(d), _p(cnt), _p(idx), k_cap, _p(small), float(h), int(order),
                            int(bool(fallback)), W, _p(cols), _p(f), _p(fii), _p(status), _p(npiv))
    return dict(cols=cols[:n], f=f[:n], fii=fii[:n], status=status[:n], npiv=npiv[:n])


def apply(n_total, gamma, diffused, w, nu_over_h2):
    g = _f64(gamma)
    d = np.zeros(max(n_total, 1), dtype=np.uint8)
    d[:len(diffused)] = diffused
    out = np.zeros(max(n_total, 1))
    cols = np.ascontiguousarray(w["cols"], dtype=np.int32)
    f = _f64(w["f"])
    fii = _f64(w["fii"])
    W = cols.shape[1] if cols.ndim == 2 else 8
    lib().orc_apply(n_total, len(g), _p(g), _p(d), _p(cols), _p(f), _p(fii), W, float(nu_over_h2), _p(out))
    return out[:n_total]


def step(x, y, gamma, h, nu, dt, r=0.5, R=2.0, c_diff=1.0, order=1, k_cap=32, max_rounds=8, fallback=True,
         fp32_search=False, capacity=None):
    """One VRM step.  Returns (x', y', gamma', stats dict)."""
    n = len(x)
    cap = capacity if capacity is not None else 2 * n + 1024
    xb = np.zeros(cap)
    yb = np.zeros(cap)
    xb[:n] = x
    yb[:n] = y
    g = _f64(gamma)
    go = np.zeros(cap)
    st = Stats()
    n2 = lib().orc_step(_p(xb), _p(yb), n, cap, _p(g), _p(go), float(h), float(r), float(R), float(nu),
                        float(c_diff), int(order), float(dt), int(k_cap), int(max_rounds), int(bool(fallback)),
                        int(bool(fp32_search)), ctypes.byref(st))
    if n2 < 0:
        raise ValueError("capacity too small: need %d" % (-n2))
    return xb[:n2].copy(), yb[:n2].copy(), go[:n2].copy(), st.as_dict()


def pipeline(x, y, gamma, h, nu, r=0.5, R=2.0, c_diff=1.0, order=1, k_cap=32, max_rounds=8, fallback=True,
             fp32_search=False):
    """Stage-by-stage run of one operator evaluation (the same steps as
    ``step``), returning every intermediate for per-stage comparisons."""
    c = constants(h, r, R, nu, c_diff, order)
    diffused = reduce(gamma, c["c_bound"])
    x2, y2, rounds, open_ = insert(x, y, diffused, h, r, R, max_rounds)
    n2 = len(x2)
    d2 = np.zeros(n2, dtype=np.uint8)
    d2[:len(x)] = diffused
    nb = neighbours(x2, y2, h, r, R, k_cap, fp32_search)
    w = solve_weights(x2, y2, d2, nb, h, order, fallback)
    dg = apply(n2, gamma, d2, w, c["nu_over_h2"])
    return dict(diffused=d2, x=x2, y=y2, rounds=rounds, open=open_, nb=nb, w=w, dgamma=dg, const=c)


# 1/k for the series below, and ln 2 split so that k * LN2_HI is exact for
# |k| < 2^20 (Cody and Waite's range reduction)
INV_K = [1.0 / k if k else 0.0 for k in range(20)]
LN2_HI = 6.93147180369123816490e-01
LN2_LO = 1.90821492927058770002e-10
INV_LN2 = 1.44269504088896338700e+00


def one_minus_exp_neg(a):
    """1 - exp(-a) for a >= 0, by a fixed sequence of separately rounded
    operations (the same on every platform): for a <= 1/4 the series
    a (1 - a/2 (1 - a/3 (... (1 - a/16)))); otherwise exp(-a) = 2^-k exp(-r),
    k = floor(a / ln 2 + 1/2), r = (a - k LN2_HI) - k LN2_LO, exp(-r) by its
    Taylor series to degree 18 in Horner form, and 1 - that; 1 for a > 700."""
    a = np.asarray(a, dtype=np.float64)
    p = np.ones_like(a)
    for k in range(16, 1, -1):
        p = 1.0 - (a * INV_K[k]) * p
    small = a * p
    ac = np.minimum(a, 700.0)
    kk = np.floor(ac * INV_LN2 + 0.5)
    r = (ac - kk * LN2_HI) - kk * LN2_LO
    q = np.ones_like(a)
    for k in range(18, 0, -1):
        q = 1.0 + ((-r) * INV_K[k] if k < len(INV_K) else (-r) / k) * q
    big = 1.0 - np.ldexp(q, -kk.astype(np.int64))
    return np.where(a <= 0.25, small, np.where(a > 700.0, 1.0, big))


def lamb_oseen_velocity(x, y, gamma, nu, t, x0=0.0, y0=0.0):
    """Azimuthal velocity of the Lamb-Oseen vortex (Sec. 5):
    u_theta = Gamma/(2 pi r) (1 - exp(-r^2/(4 nu t))), as
    (u, v) = (-(y - y0), x - x0) * k with k = Gamma/(2 pi r^2) * one_minus_exp_neg(r^2/(4 nu t));
    products and sums rounded separately, k = 0 at r = 0."""
    dx = np.asarray(x, dtype=np.float64) - x0
    dy = np.asarray(y, dtype=np.float64) - y0
    r2 = dx * dx + dy * dy
    with np.errstate(divide="ignore", invalid="ignore"):
        a = r2 / ((4.0 * nu) * t)
        k = (gamma / ((2.0 * np.pi) * r2)) * one_minus_exp_neg(a)
    k = np.where(r2 > 0.0, k, 0.0)
    return -dy * k, dx * k


def rk3_step(x, y, gamma, h, nu, t, dt, vel=None, r=0.5, R=2.0, c_diff=1.0, order=1, k_cap=32, max_rounds=8,
             fallback=True):
    """One SSP-RK3 (Shu-Osher) step of dx/dt = u(x, t), dGamma/dt = L(x) Gamma
    (the reduced operator of Sec. 3.5 with the diffused set fixed at the start
    of the step): growth control and insertion once on the step's initial
    cloud, neighbourhoods and weights at every stage's positions.
        X1 = X0 + dt u(X0, t),           G1 = G0 + dt L(X0) G0
        X2 = 3/4 X0 + 1/4 (X1 + dt u(X1, t + dt)),   G2 likewise with L(X1) G1
        X3 = 1/3 X0 + 2/3 (X2 + dt u(X2, t + dt/2)), G3 likewise with L(X2) G2
    vel: dict(gamma, nu, x0, y0) of the Lamb-Oseen field, dict(eps=...) for
    the particles' own smoothed Biot-Savart velocity (direct sum, stage
    circulations), or None (no advection: the positions stay those of the
    start).  Products and sums rounded separately.  Returns (x', y',
    gamma', stats)."""
    c = constants(h, r, R, nu, c_diff, order)
    n = len(x)
    diffused = reduce(gamma, c["c_bound"])
    X0, Y0, rounds, open_ = insert(x, y, diffused, h, r, R, max_rounds)
    n2 = len(X0)
    d2 = np.zeros(n2, dtype=np.uint8)
    d2[:n] = diffused
    G0 = np.zeros(n2)
    G0[:n] = gamma
    third, two_thirds = 1.0 / 3.0, 2.0 / 3.0
    coef = [(None, None), (0.75, 0.25), (third, two_thirds)]
    times = [t, t + dt, t + 0.5 * dt]
    Xs, Ys, Gs = X0, Y0, G0
    stats = dict(n_in=n, n_out=n2, n_diffused=int(diffused.sum()), n_inserted=n2 - n, rounds=rounds,
                 small_ok=0, full_ok=0, no_stencil=0)
    for s in range(3):
        nb = neighbours(Xs, Ys, h, r, R, k_cap)
        w = solve_weights(Xs, Ys, d2, nb, h, order, fallback)
        stats["small_ok"] += int(np.sum(w["status"] == 1))
        stats["full_ok"] += int(np.sum(w["status"] == 2))
        stats["no_stencil"] += int(np.sum(w["status"] == 3))
        dg = apply(n2, Gs, d2, w, c["nu_over_h2"])
        Ge = Gs + dt * dg
        if vel is not None:
            if "eps" in vel:
                u, v = biot_savart(Xs, Ys, Gs, Xs, Ys, vel["eps"])
            else:
                u, v = lamb_oseen_velocity(Xs, Ys, vel["gamma"], vel["nu"], times[s], vel.get("x0", 0.0),
                                           vel.get("y0", 0.0))
            Xe = Xs + dt * u
            Ye = Ys + dt * v
        if s == 0:
            Gs = Ge
            if vel is not None:
                Xs, Ys = Xe, Ye
        else:
            a, b = coef[s]
            Gs = a * G0 + b * Ge
            if vel is not None:
                Xs = a * X0 + b * Xe
                Ys = a * Y0 + b * Ye
    return Xs, Ys, Gs, stats


def biot_savart(xs, ys, gamma, xt, yt, eps, block=2048):
    """Smoothed Biot-Savart velocity at the targets (Sec. 5, Eq. smoothkernel):
    u_h(x) = sum_j Gamma_j K_eps(x - x_j),
    K_eps(x) = (-y, x) / (2 pi |x|^2) (1 - exp(-|x/eps|^2)),  K_eps(0) = 0;
    direct sum in FP64 (1 - exp(-q) as -expm1(-q)), targets in blocks."""
    xs = np.asarray(xs, dtype=np.float64)
    ys = np.asarray(ys, dtype=np.float64)
    g = np.asarray(gamma, dtype=np.float64)
    xt = np.asarray(xt, dtype=np.float64)
    yt = np.asarray(yt, dtype=np.float64)
    u = np.zeros(len(xt))
    v = np.zeros(len(xt))
    for a in range(0, len(xt), block):
        dx = xt[a:a + block, None] - xs[None, :]
        dy = yt[a:a + block, None] - ys[None, :]
        r2 = dx * dx + dy * dy
        with np.errstate(divide="ignore", invalid="ignore"):
            k = np.where(r2 > 0.0, -np.expm1(-r2 / (eps * eps)) / ((2.0 * np.pi) * r2), 0.0)
        u[a:a + block] = -(dy * k) @ g
        v[a:a + block] = (dx * k) @ g
    return u, v



def remove_close(x, y, gamma, h, r=0.5, R=2.0):
    """Particle removal (outlook of Sec. 6.2): returns (x', y', gamma', removed
    flags, number of candidates, stencils dict(cols, w) [n x 4], close flags)."""
    x, y, g = _f64(x), _f64(y), _f64(gamma)
    n = len(x)
    m = max(n, 1)
    xo, yo, go = np.zeros(m), np.zeros(m), np.zeros(m)
    removed = np.zeros(m, dtype=np.uint8)
    cand = ctypes.c_long(0)
    k = lib().orc_remove(_p(x), _p(y), _p(g), n, float(h), float(r), float(R), _p(xo), _p(yo), _p(go), _p(removed),
                         ctypes.byref(cand))
    rh, Rh = r * h, R * h
    close = np.zeros(m, dtype=np.uint8)
    lib().orc_close(_p(x), _p(y), _p(g), n, rh * rh, Rh, _p(close))
    cols = np.full((m, 4), -1, dtype=np.int32)
    w = np.zeros((m, 4))
    rem2 = np.zeros(m, dtype=np.uint8)
    lib().orc_remove_weights(_p(x), _p(y), n, _p(close), float(h), rh * rh, Rh * Rh, Rh, _p(rem2), _p(cols), _p(w))
    return (xo[:k].copy(), yo[:k].copy(), go[:k].copy(), removed[:n].copy(), cand.value,
            dict(cols=cols[:n], w=w[:n]), close[:n].copy())
