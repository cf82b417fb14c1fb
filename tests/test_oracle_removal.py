"""Pins of the oracle's particle removal (the outlook of Sec. 6.2: a particle
that came too close to another is redistributed to its neighbours by an
approximation of the identity operator and removed).

* Candidates against an O(n^2) brute force: a particle closer than r h to one
  of larger key (|Gamma|, index).
* Every removed particle's weights meet the identity's conditions that
  non-negative weights can meet (sum g = 1, sum g r = 0, g >= 0) and land on
  kept annulus neighbours; conservation of circulation and of its first
  moments over the whole pass.
* Completeness: a candidate stays exactly when the origin is outside the
  convex hull of its kept small neighbourhood (vertex enumeration over all
  triangles, segments and points of the columns).
* Kept particles keep their positions, in index order.
"""
import itertools

import numpy as np
import pytest

import vrm_inputs


def crowded_cloud(n=1600, h=0.02, extra=0.1, seed=3):
    """Jittered lattice plus a fraction `extra` of particles placed within
    0.3 h of existing ones (seeded)."""
    x, y, g = vrm_inputs.random_cloud(n, h=h, jitter=0.3, seed=seed)
    rng = np.random.default_rng(seed + 100)
    m = int(extra * len(x))
    k = rng.choice(len(x), m, replace=False)
    x2 = np.concatenate([x, x[k] + rng.uniform(-0.3, 0.3, m) * h])
    y2 = np.concatenate([y, y[k] + rng.uniform(-0.3, 0.3, m) * h])
    g2 = np.concatenate([g, g[k] * rng.uniform(-1, 1, m)])
    return x2, y2, g2, h


def brute_candidates(x, y, g, rh):
    n = len(x)
    a = np.abs(g)
    out = np.zeros(n, dtype=np.uint8)
    for i in range(n):
        d2 = (x - x[i]) * (x - x[i]) + (y - y[i]) * (y - y[i])
        for j in np.nonzero(d2 < rh * rh)[0]:
            if j != i and (a[i] < a[j] or (a[i] == a[j] and i < j)):
                out[i] = 1
                break
    return out


@pytest.mark.parametrize("seed", [3, 4])
def test_candidates_brute_force(orc, seed):
    x, y, g, h = crowded_cloud(900, seed=seed)
    *_, cand, _, close = orc.remove_close(x, y, g, h)
    assert np.array_equal(close, brute_candidates(x, y, g, 0.5 * h))
    assert cand == int(close.sum()) > 0


def kept_small(x, y, i, close, h, r=0.5, R=2.0):
    """Closest kept particle of every 45-degree segment of i's annulus
    (segments from atan2, independent of the oracle's comparisons)."""
    dx, dy = x - x[i], y - y[i]
    d2 = dx * dx + dy * dy
    ang = np.arctan2(dy, dx) % (2 * np.pi)
    seg = np.floor(ang / (np.pi / 4)).astype(int) % 8
    best = {}
    for j in np.nonzero((d2 >= (r * h) ** 2) & (d2 <= (R * h) ** 2))[0]:
        if j == i or close[j]:
            continue
        s = seg[j]
        if s not in best or (d2[j], j) < (d2[best[s]], best[s]):
            best[s] = j
    return sorted(best.values())


def origin_in_hull(px, py):
    # some point, segment or triangle of the columns holds the origin with
    # non-negative barycentric weights
    pts = list(zip(px, py))
    for k in (1, 2, 3):
        for S in itertools.combinations(range(len(pts)), k):
            A = np.array([[1.0] * k, [pts[s][0] for s in S], [pts[s][1] for s in S]])
            w, res, rank, _ = np.linalg.lstsq(A, np.array([1.0, 0.0, 0.0]), rcond=None)
            if rank == k and np.all(w >= -1e-9) and np.max(np.abs(A @ w - [1, 0, 0])) < 1e-9:
                return True
    return False


@pytest.mark.parametrize("seed", [3, 5])
def test_identity_stencils_and_conservation(orc, seed):
    x, y, g, h = crowded_cloud(1600, seed=seed)
    xo, yo, go, removed, cand, st, close = orc.remove_close(x, y, g, h)
    n = len(x)
    assert removed.sum() > 0 and len(xo) == n - removed.sum()
    # every removed particle was a candidate; its stencil meets the identity's
    # conditions on kept annulus neighbours
    assert np.all(close[removed == 1] == 1)
    for i in np.nonzero(removed)[0]:
        c = st["cols"][i]
        w = st["w"][i][c >= 0]
        js = c[c >= 0]
        assert len(js) >= 1 and np.all(w > 0)
        assert not np.any(close[js])
        d2 = (x[js] - x[i]) ** 2 + (y[js] - y[i]) ** 2
        assert np.all(d2 >= (0.5 * h) ** 2) and np.all(d2 <= (2 * h) ** 2)
        xi, eta = (x[js] - x[i]) / h, (y[js] - y[i]) / h
        assert abs(np.sum(w) - 1.0) < 1e-12
        assert abs(np.sum(w * xi)) < 1e-12 and abs(np.sum(w * eta)) < 1e-12
    # circulation and its first moments conserved
    scale = np.sum(np.abs(g))
    assert abs(go.sum() - g.sum()) <= 1e-14 * scale
    assert abs(np.sum(go * xo) - np.sum(g * x)) <= 1e-13 * scale
    assert abs(np.sum(go * yo) - np.sum(g * y)) <= 1e-13 * scale
    # kept particles keep their positions, in index order
    keep = np.nonzero(removed == 0)[0]
    assert np.array_equal(xo, x[keep]) and np.array_equal(yo, y[keep])


def test_candidate_stays_iff_origin_outside_hull(orc):
    x, y, g, h = crowded_cloud(900, seed=6)
    _, _, _, removed, _, _, close = orc.remove_close(x, y, g, h)
    stayed = 0
    for i in np.nonzero(close)[0]:
        js = kept_small(x, y, i, close, h)
        inside = origin_in_hull((x[js] - x[i]) / h, (y[js] - y[i]) / h) if js else False
        assert bool(removed[i]) == inside, i
        stayed += not inside
    assert stayed > 0  # the cloud's edge: some candidates have no stencil


def test_single_extra_particle(orc):
    # a lattice with one extra particle 0.1 h east of a lattice point: the
    # extra one (smaller |Gamma|) goes, the lattice point keeps its value,
    # and the extra circulation lands on the ring around
    h = 1.0 / 32
    x, y = vrm_inputs.lattice(h, -0.5, 0.5)
    n = len(x)
    g = np.full(n, 1e-3)
    c = np.argmin(x * x + y * y)
    x = np.append(x, x[c] + 0.1 * h)
    y = np.append(y, y[c])
    g = np.append(g, 2e-4)
    xo, yo, go, removed, cand, st, close = orc.remove_close(x, y, g, h)
    assert cand == 1 and removed[n] == 1 and removed.sum() == 1
    assert go[c] == g[c]
    moved = go - g[:n]
    assert abs(moved.sum() - 2e-4) < 1e-18
    assert abs(np.sum(moved * x[:n]) - 2e-4 * x[n]) < 1e-18


def test_empty_and_no_candidates(orc):
    xo, yo, go, removed, cand, _, _ = orc.remove_close(np.zeros(0), np.zeros(0), np.zeros(0), 0.1)
    assert len(xo) == 0 and cand == 0
    h = 1.0 / 16
    x, y = vrm_inputs.lattice(h, -0.5, 0.5)
    g = np.linspace(1, 2, len(x))
    xo, yo, go, removed, cand, _, _ = orc.remove_close(x, y, g, h)
    assert cand == 0 and np.array_equal(go, g) and np.array_equal(xo, x)
