"""Pins of the oracle's geometry: segments, neighbourhoods, insertion.

Each check compares the oracle with something other than itself: atan2
angles, brute-force distance tests in numpy, and the paper's insertion
geometry (Sec. 4.2, Fig. insertion).
"""
import math

import numpy as np
import pytest

import vrm_inputs


def test_segment_matches_atan2_away_from_rays(orc):
    rng = np.random.default_rng(1)
    pts = rng.standard_normal((4000, 2))
    for dx, dy in pts:
        ang = math.atan2(dy, dx) % (2 * math.pi)
        k = ang / (math.pi / 4)
        if abs(k - round(k)) < 1e-9:
            continue
        assert orc.segment(dx, dy) == int(math.floor(k)) % 8


def test_segment_half_open_rays_and_antisymmetry(orc):
    # ray k*45deg belongs to segment k (half-open [k pi/4, (k+1) pi/4))
    rays = [(1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1)]
    for k, (dx, dy) in enumerate(rays):
        assert orc.segment(dx, dy) == k
    rng = np.random.default_rng(2)
    pts = np.concatenate([rng.standard_normal((2000, 2)), np.array(rays, float) * 0.3])
    for dx, dy in pts:
        assert orc.segment(-dx, -dy) == (orc.segment(dx, dy) + 4) % 8


def brute_neighbours(x, y, lo2, hi2, fp32=False):
    if fp32:
        xf, yf = x.astype(np.float32), y.astype(np.float32)
        dx = xf[None, :] - xf[:, None]
        dy = yf[None, :] - yf[:, None]
        d2 = dx * dx + dy * dy
        ok = (d2 >= np.float32(lo2)) & (d2 <= np.float32(hi2))
    else:
        dx = x[None, :] - x[:, None]
        dy = y[None, :] - y[:, None]
        d2 = dx * dx + dy * dy
        ok = (d2 >= lo2) & (d2 <= hi2)
    np.fill_diagonal(ok, False)
    return ok, d2.astype(np.float64), dx.astype(np.float64), dy.astype(np.float64)


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("seed,kind", [(0, "lattice"), (1, "lattice"), (2, "scatter"), (3, "scatter")])
def test_neighbours_match_brute_force(orc, fp32, seed, kind):
    h = 0.05
    if kind == "lattice":
        x, y, _ = vrm_inputs.random_cloud(900, h=h, jitter=0.35, seed=seed)
    else:
        x, y, _ = vrm_inputs.uniform_scatter(700, half_width=0.7, seed=seed)
    c = orc.constants(h)
    nb = orc.neighbours(x, y, h, k_cap=64, fp32=fp32)
    ok, d2, dx, dy = brute_neighbours(x, y, c["lo2"], c["hi2"], fp32)
    ang = np.arctan2(dy, dx) % (2 * np.pi)
    for i in range(len(x)):
        js = np.nonzero(ok[i])[0]
        assert nb["count"][i] == len(js)
        assert list(nb["idx"][i, :len(js)]) == list(js)
        # segments from atan2 angles (independent of the comparison-based
        # classifier); random clouds put no point on a ray
        m = 0
        segs = np.floor(ang[i, js] / (np.pi / 4)).astype(int) % 8
        on_ray = np.abs(ang[i, js] / (np.pi / 4) - np.round(ang[i, js] / (np.pi / 4))) < 1e-9
        assert not on_ray.any()
        for s in set(segs):
            m |= 1 << int(s)
        assert nb["mask"][i] == m
        for s in range(8):
            cand = js[segs == s]
            if len(cand) == 0:
                assert nb["small"][i, s] == -1
            else:
                dd = d2[i, cand]
                best = cand[np.lexsort((cand, dd))[0]]
                assert nb["small"][i, s] == best


def test_neighbours_ties_and_lattice(orc):
    # perfect lattice with binary-exact coordinates (h = 1/8): equal
    # distances everywhere, the annulus ends are inclusive, ties go to the
    # lower index
    h = 0.125
    x, y = vrm_inputs.lattice(h, -0.625, 0.625)
    nb = orc.neighbours(x, y, h)
    side = 11
    i = 5 * side + 5  # centre
    # annulus [0.5h, 2h]: offsets with 0.25 <= a^2+b^2 <= 4
    expect = sorted((5 + b) * side + (5 + a) for a in range(-2, 3) for b in range(-2, 3)
                    if 0.25 <= a * a + b * b <= 4)
    assert list(nb["idx"][i, :nb["count"][i]]) == expect
    assert nb["count"][i] == 12
    # small neighbourhood: E, NE, N, NW, W, SW, S, SE in segments 0..7
    off = [(1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1)]
    assert list(nb["small"][i]) == [(5 + b) * side + (5 + a) for a, b in off]


def test_empty_and_single(orc):
    nb = orc.neighbours(np.zeros(0), np.zeros(0), 0.1)
    assert nb["max_count"] == 0
    nb = orc.neighbours(np.zeros(1), np.zeros(1), 0.1)
    assert nb["count"][0] == 0 and nb["mask"][0] == 0 and (nb["small"][0] == -1).all()


def test_insertion_single_particle_geometry(orc):
    # Sec. 5 starts from one Dirac: all 8 segments are empty, so the 8 points
    # at radius 1.5h on the segment centre lines are inserted (Sec. 4.2).
    h = 0.1
    x2, y2, rounds, open_ = orc.insert(np.array([0.3]), np.array([-0.2]), np.array([1], np.uint8), h)
    assert len(x2) == 9 and rounds == 1 and open_ == 0
    for s in range(8):
        th = (s + 0.5) * math.pi / 4
        assert abs(x2[1 + s] - (0.3 + 1.5 * h * math.cos(th))) < 1e-15
        assert abs(y2[1 + s] - (-0.2 + 1.5 * h * math.sin(th))) < 1e-15


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_insertion_fills_segments_and_keeps_separation(orc, seed):
    # After insertion every diffused particle has all 8 segments occupied and
    # no inserted point lies closer than r h to any other point (Sec. 4.2).
    h = 0.05
    x, y, g = vrm_inputs.uniform_scatter(150, half_width=0.5, seed=seed)
    d = np.ones(len(x), np.uint8)
    d[::3] = 0
    x2, y2, rounds, open_ = orc.insert(x, y, d, h, max_rounds=16)
    assert open_ == 0
    assert len(x2) > len(x)
    nb = orc.neighbours(x2, y2, h, k_cap=64)
    for i in range(len(x)):
        if d[i]:
            assert nb["mask"][i] == 0xFF
    n = len(x)
    rh2 = (0.5 * h) ** 2
    dx = x2[n:, None] - x2[None, :]
    dy = y2[n:, None] - y2[None, :]
    d2 = dx * dx + dy * dy
    for a in range(len(x2) - n):
        d2[a, n + a] = np.inf
    assert (d2 >= rh2 * (1 - 1e-12)).all()


def test_insertion_keeps_full_lattice(orc):
    # an interior point of a binary-exact lattice already has all segments
    # occupied (the diagonal neighbours sit on the rays k pi/4 and belong to
    # segment k)
    h = 0.125
    x, y = vrm_inputs.lattice(h, -0.625, 0.625)
    d = np.zeros(len(x), np.uint8)
    d[5 * 11 + 5] = 1
    x2, _, rounds, _ = orc.insert(x, y, d, h)
    assert len(x2) == len(x) and rounds == 0
