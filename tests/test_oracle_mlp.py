"""Pins of the learned-proposal oracle (oracle/mlp.py) against what the
mathematics fixes: closed forms, finite differences, library routines
(torch's bfloat16 rounding and AdamW, numpy's least squares) and the paper's
single-particle example (Sec. 5: eight inserted neighbours at 1.5h)."""
import math

import numpy as np
import pytest

from oracle import mlp

torch = pytest.importorskip("torch")


def test_parameter_count():
    # 96*256 + 256 + 2 * (256*256 + 256) + 256*32 + 32
    assert mlp.N_PARAMS == 164640
    theta = np.arange(mlp.N_PARAMS, dtype=np.float64)
    assert np.array_equal(mlp.flatten(mlp.unflatten(theta)), theta)
    W1, b1 = mlp.unflatten(theta)[0]
    assert W1.shape == (256, 96) and b1[0] == 256 * 96


def test_bf16_rounding():
    assert mlp.to_bf16(1.0) == 1.0
    assert mlp.to_bf16(1.0 + 2.0 ** -8) == 1.0  # tie to even
    assert mlp.to_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie to even (upwards)
    assert mlp.to_bf16(-2.0 ** -130) == -2.0 ** -130 or mlp.to_bf16(-2.0 ** -130) <= 0
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-3, 5000), rng.normal(0, 1e4, 5000)])
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.to_bf16(a), ref)


def test_gelu_closed_forms():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    # tanh form at 1: 0.5 (1 + tanh(sqrt(2/pi) 1.044715)) = 0.8411919906082768; it
    # stays within 2e-4 of the erf form Phi(1) = 0.8413447460685429
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.5 * (1 + math.tanh(math.sqrt(2 / math.pi) * 1.044715))) < 1e-15
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 2e-4
    assert abs(mlp.gelu(np.array([-1.0]))[0] + 0.15865525393145707) < 2e-4
    # odd part: gelu(z) - gelu(-z) = z
    z = np.linspace(-5, 5, 101)
    assert np.max(np.abs(mlp.gelu(z) - mlp.gelu(-z) - z)) < 1e-14
    assert abs(mlp.gelu(np.array([12.0]))[0] - 12.0) < 1e-12 and abs(mlp.gelu(np.array([-12.0]))[0]) < 1e-12
    z = np.linspace(-6, 6, 241)
    e = 1e-6
    fd = (mlp.gelu(z + e) - mlp.gelu(z - e)) / (2 * e)
    assert np.max(np.abs(fd - mlp.gelu_grad(z))) < 1e-8


def small_problem(seed=0, B=6):
    rng = np.random.default_rng(seed)
    theta = np.concatenate([np.concatenate([rng.normal(0, 1 / math.sqrt(i), o * i), rng.normal(0, 0.1, o)])
                            for o, i in mlp.SHAPES])
    X = rng.normal(0, 1, (B, mlp.N_IN))
    T = rng.normal(0, 0.3, (B, mlp.N_OUT))
    M = (rng.random((B, mlp.N_OUT)) < 0.6).astype(np.float64)
    return theta, X, T, M


def test_backward_matches_central_differences():
    theta, X, T, M = small_problem()
    Y, cache = mlp.forward(theta, X)
    L, dY = mlp.loss(Y, T, M)
    g = mlp.backward(theta, cache, dY)
    rng = np.random.default_rng(1)
    # one index in every weight block and bias block of every layer, plus random ones
    offs, o = [], 0
    for rows, cols in mlp.SHAPES:
        offs += [o + int(rng.integers(rows * cols)), o + rows * cols + int(rng.integers(rows))]
        o += rows * cols + rows
    offs += list(rng.integers(0, mlp.N_PARAMS, 40))
    for k in offs:
        e = 1e-5 * max(1.0, abs(theta[k]))
        tp, tm = theta.copy(), theta.copy()
        tp[k] += e
        tm[k] -= e
        Lp = mlp.loss(mlp.forward(tp, X)[0], T, M)[0]
        Lm = mlp.loss(mlp.forward(tm, X)[0], T, M)[0]
        fd = (Lp - Lm) / (2 * e)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(fd), 1e-3), (k, fd, g[k])


def test_loss_is_a_masked_mean():
    Y = np.array([[1.0, 2.0, 3.0]])
    T = np.array([[0.0, 0.0, 0.0]])
    M = np.array([[1.0, 0.0, 1.0]])
    L, dY = mlp.loss(Y, T, M)
    assert L == (1.0 + 9.0) / 2 and np.array_equal(dY, [[1.0, 0.0, 3.0]])


def test_adamw_matches_torch():
    rng = np.random.default_rng(2)
    theta = rng.normal(0, 1, 1000)
    grads = [rng.normal(0, 1, 1000) for _ in range(5)]
    hp = dict(lr=3e-3, beta1=0.9, beta2=0.99, eps=1e-8, weight_decay=0.01)
    p = torch.nn.Parameter(torch.from_numpy(theta.copy()))
    opt = torch.optim.AdamW([p], lr=hp["lr"], betas=(hp["beta1"], hp["beta2"]), eps=hp["eps"],
                            weight_decay=hp["weight_decay"])
    th, m, v = theta.copy(), np.zeros(1000), np.zeros(1000)
    for t, g in enumerate(grads, start=1):
        p.grad = torch.from_numpy(g.copy())
        opt.step()
        th, m, v = mlp.adamw(th, g, m, v, t, **hp)
    # torch decays the weights before the Adam update (theta (1 - lr wd)); the
    # oracle applies lr (update + wd theta): identical to first order in lr wd
    assert np.max(np.abs(p.detach().numpy() - th)) < 1e-6
    # first step in closed form: m^ = g, v^ = g^2
    th1, _, _ = mlp.adamw(theta, grads[0], np.zeros(1000), np.zeros(1000), 1, lr=1e-3, eps=0.0)
    assert np.allclose(th1, theta - 1e-3 * np.sign(grads[0]), rtol=0, atol=1e-15)


def test_segments_and_feature_slots():
    # unit lattice around the origin: E NE N NW W SW S SE fall in segments 0..7
    off = [(1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1)]
    assert [mlp.segment(dx, dy) for dx, dy in off] == list(range(8))
    h = 0.5
    x = np.array([0.0] + [h * a for a, _ in off] + [2 * h, 1.5 * h])
    y = np.array([0.0] + [h * b for _, b in off] + [0.0, 0.25 * h])
    row = list(range(10, 0, -1))  # any order
    X, slots = mlp.features(x, y, h, 0, row)
    # segment 0 holds E (d2 = h^2), (1.5h, 0.25h) (d2 = 2.3125 h^2) and (2h, 0) (4 h^2), in that order
    assert list(slots[:3]) == [1, 10, 9] and list(slots[3:10]) == [2, 3, 4, 5, 6, 7, 8]
    assert np.all(slots[10:] == -1)
    assert X[0] == 1.0 and X[1] == 1.5 and X[2] == 2.0 and X[32] == 0.0 and X[33] == 0.25
    assert np.array_equal(X[64:74], np.ones(10)) and np.all(X[74:] == 0)


def test_support_selection():
    f0 = np.zeros(32, dtype=np.float32)
    slots = np.arange(32)
    f0[[3, 5, 7, 9, 11, 13, 15, 17, 19, 21]] = [0.5, 0.9, 0.1, 0.9, 0.2, 0.3, 0.4, 0.05, 0.6, 0.7]
    assert mlp.support(f0, slots) == [3, 5, 9, 11, 13, 15, 19, 21]
    slots[5] = -1  # empty slots never enter
    assert 5 not in mlp.support(f0, slots)
    f0[:] = -1.0
    assert mlp.support(f0, np.arange(32)) == []


def test_projection_least_change():
    rng = np.random.default_rng(3)
    for _ in range(50):
        K = int(rng.integers(5, 9))
        ang = rng.uniform(0, 2 * math.pi, K)
        rad = rng.uniform(0.5, 2.0, K)
        xi, eta = rad * np.cos(ang), rad * np.sin(ang)
        V = mlp.vandermonde(xi, eta)
        cond = np.linalg.cond(V @ V.T)
        if cond > 1e5:  # ill-conditioned supports fail the residual check and go to the LP
            continue
        f0 = rng.uniform(0, 1, K)
        f, res = mlp.project(xi, eta, f0)
        assert res <= 1e-12
        # the correction is the minimum-norm solution of V d = b - V f0
        d_ref = np.linalg.lstsq(V, mlp.B_RHS - V @ f0, rcond=None)[0]
        assert np.max(np.abs((f - f0) - d_ref)) < 1e-10
        # a proposal that already meets the conditions is left alone
        f2, _ = mlp.project(xi, eta, f)
        assert np.max(np.abs(f2 - f)) < 1e-15 * cond * max(1.0, np.max(np.abs(f)))  # eps * condition


def test_projection_single_particle_example():
    # Sec. 5: a lone particle gets 8 inserted neighbours at 1.5h on the segment
    # centre lines; every stencil meeting the moment conditions has
    # sum f~ = 4 / 1.5^2 = 16/9 (rows (2,0) + (0,2) with |xi|^2 = 2.25)
    ang = (np.arange(8) + 0.5) * math.pi / 4
    xi, eta = 1.5 * np.cos(ang), 1.5 * np.sin(ang)
    rng = np.random.default_rng(4)
    for _ in range(20):
        f, res = mlp.project(xi, eta, rng.uniform(0, 1, 8))
        assert res <= 1e-12 and abs(np.sum(f) - 16.0 / 9.0) < 1e-13
    # the symmetric proposal projects to the uniform stencil 2/9
    f, _ = mlp.project(xi, eta, np.full(8, 0.3))
    assert np.max(np.abs(f - 2.0 / 9.0)) < 1e-14


def lattice8():
    off = [(1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1)]
    x = np.array([0.0] + [a for a, _ in off])
    y = np.array([0.0] + [b for _, b in off])
    slots = np.full(32, -1)
    slots[:8] = np.arange(1, 9)
    return x, y, slots


def test_learned_stencil_accepts_valid_and_rejects_infeasible():
    # unit lattice neighbours, the 5-point stencil proposal (f~ = 1 on E N W S)
    # plus a little weight on the diagonals: the top five slots (E N W S and
    # the first diagonal) solve square to the 5-point stencil, whose zero
    # weight on the diagonal is not kept
    h = 1.0
    x, y, slots = lattice8()
    f0 = np.zeros(32, dtype=np.float32)
    f0[:8] = [1, 0.01, 1, 0.01, 1, 0.01, 1, 0.01]
    ok, js, f, fii, tried = mlp.learned_stencil(x, y, h, 0, slots, f0, trials=True)
    assert ok and tried == 1 and js == [1, 3, 5, 7] and np.all(f == 1.0) and fii == -4.0
    # the diagonals and W: the square system gives the rotated 5-point stencil
    f0[:8] = [0.0, 1.0, 0.0, 1.0, 3.0, 1.0, 0.0, 1.0]
    ok, js, f, _ = mlp.learned_stencil(x, y, h, 0, slots, f0)
    assert ok and js == [2, 4, 6, 8] and np.allclose(f, 0.5, rtol=0, atol=1e-15)
    # neighbours in the upper half plane only: sum f eta = 0 forces f = 0 on
    # them, no support passes (Sec. 4.2's motive for insertion)
    up = [k for k in range(1, 9) if y[k] > 0] + [k for k in range(1, 9) if y[k] == 0]
    sl = np.full(32, -1)
    sl[:len(up)] = up
    ok, _, _, _, tried = mlp.learned_stencil(x, y, h, 0, sl, np.ones(32, np.float32), trials=True)
    assert not ok and tried == 1  # five candidates: one support
    # fewer than five candidates: nothing to solve
    sl = np.full(32, -1)
    sl[:4] = [1, 3, 5, 7]
    ok, _, _, _, tried = mlp.learned_stencil(x, y, h, 0, sl, np.ones(32, np.float32), trials=True)
    assert not ok and tried == 0


def test_first_passing_support_in_subset_order():
    # jittered rings of 8 candidates, weights well away from zero on every
    # support (so the binary32 screen and the FP64 test agree): the chosen
    # support is the first one, in subset_order, whose exact solution is
    # non-negative (brute force with numpy's solver)
    rng = np.random.default_rng(31)
    seen = 0
    for case in range(200):
        th = np.arange(8) * np.pi / 4 + rng.uniform(0, np.pi / 4, 8)
        rad = rng.uniform(0.6, 1.9, 8)
        x = np.concatenate([[0.0], rad * np.cos(th)])
        y = np.concatenate([[0.0], rad * np.sin(th)])
        slots = np.full(32, -1)
        slots[:8] = np.arange(1, 9)
        f0 = np.zeros(32, dtype=np.float32)
        f0[:8] = rng.uniform(0, 1, 8)
        ranked = mlp.candidates(f0, slots)
        expect, margin_ok = None, True
        for sub in mlp.subset_order(8):
            S = sorted(ranked[r] for r in sub)
            V = mlp.vandermonde(x[slots[S]], y[slots[S]])
            if abs(np.linalg.det(V)) < 1e-9:
                continue
            f = np.linalg.solve(V, mlp.B_RHS)
            if np.min(np.abs(f)) < 1e-5:
                margin_ok = False
                break
            if np.all(f > 0):
                expect = [int(slots[k]) for k in S]
                break
        if not margin_ok:
            continue
        seen += 1
        ok, js, f, _ = mlp.learned_stencil(x, y, 1.0, 0, slots, f0)
        assert ok == (expect is not None) and (not ok or js == expect), case
    assert seen > 150


@pytest.mark.parametrize("seed", range(30))
def test_support_search_finds_a_stencil_iff_the_lp_does(orc, seed):
    # every feasible LP on the eight columns has a basic feasible solution
    # on five of them, so searching all supports is complete: the learned
    # stencil exists exactly when the oracle's phase-I simplex finds one
    rng = np.random.default_rng(400 + seed)
    th = np.arange(8) * np.pi / 4 + rng.uniform(0, np.pi / 4, 8)
    if seed % 3 == 0:
        th = rng.uniform(0, 1.6 * np.pi, 8)  # some with an open sector
    rad = rng.uniform(0.5, 2.0, 8)
    x = np.concatenate([[0.0], rad * np.cos(th)])
    y = np.concatenate([[0.0], rad * np.sin(th)])
    slots = np.full(32, -1)
    slots[:8] = np.arange(1, 9)
    f0 = np.zeros(32, dtype=np.float32)
    f0[:8] = rng.uniform(0, 1, 8)
    ok, js, f, _ = mlp.learned_stencil(x, y, 1.0, 0, slots, f0)
    st, _, _, _ = orc.phase1(orc.vandermonde(1, x[1:], y[1:]), mlp.B_RHS)
    assert ok == (st == 0)
    if ok:
        V = mlp.vandermonde(x[js], y[js])
        assert np.all(f > 0) and np.max(np.abs(V @ f - mlp.B_RHS)) <= 1e-12


def test_subset_order():
    from math import comb
    for nc in range(5, 9):
        order = mlp.subset_order(nc)
        assert len(order) == len(set(order)) == comb(nc, 5)
        assert order[0] == (0, 1, 2, 3, 4)
        sums = [sum(r) for r in order]
        assert sums == sorted(sums)
    assert mlp.subset_order(4) == []


def test_nearly_dependent_rows_reject():
    # four neighbours on one line plus one: rows (1,0) and (2,0) ... leave the
    # five columns dependent in (0,1)/(1,1)/(0,2); no support solves
    xl = np.array([0.0, 1.0, 2.0, -1.0, -2.0, 0.0])
    yl = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 1.0])
    sl = np.full(32, -1)
    sl[:5] = np.arange(1, 6)
    f0l = np.zeros(32, dtype=np.float32)
    f0l[:5] = 1.0
    ok, _, _, _ = mlp.learned_stencil(xl, yl, 1.0, 0, sl, f0l)
    assert not ok
    assert not mlp.gram_ok(mlp.vandermonde(xl[1:], yl[1:]))


def test_square_solve_is_gaussian_elimination():
    rng = np.random.default_rng(7)
    for _ in range(50):
        V = rng.normal(0, 1, (5, 5))
        b = rng.normal(0, 1, 5)
        f = mlp.square_solve(V, b)
        assert np.allclose(f, np.linalg.solve(V, b), rtol=1e-10, atol=1e-12)
    # a zero column is singular
    V = rng.normal(0, 1, (5, 5))
    V[:, 2] = 0.0
    assert mlp.square_solve(V, np.ones(5)) is None


def test_square_solve32_is_binary32_elimination():
    # well-conditioned jittered supports: within binary32 accuracy of the
    # exact solution; the 5-point supports are exact in binary32
    rng = np.random.default_rng(8)
    for _ in range(200):
        th = np.arange(5) * 2 * np.pi / 5 + rng.uniform(-0.3, 0.3, 5)
        rad = rng.uniform(0.7, 1.8, 5)
        xi, eta = rad * np.cos(th), rad * np.sin(th)
        V = mlp.vandermonde(xi, eta)
        if np.linalg.cond(V) > 1e3:
            continue
        f = np.linalg.solve(V, mlp.B_RHS)
        f32 = mlp.square_solve32(xi, eta)
        assert f32.dtype == np.float32
        assert np.max(np.abs(f32 - f)) <= 1e-4 * np.max(np.abs(f))
    f32 = mlp.square_solve32(np.array([1.0, 1.0, 0.0, -1.0, 0.0]), np.array([0.0, 1.0, 1.0, 0.0, -1.0]))
    assert np.array_equal(f32, np.array([1, 0, 1, 1, 1], np.float32))
    # a repeated column is singular
    assert mlp.square_solve32(np.array([1.0, 1.0, 0.0, -1.0, 0.0]), np.array([0.0, 0.0, 1.0, 0.0, -1.0])) is None


def test_top_five_basis_gives_the_vertex():
    # E, N, W, S and NE on the unit lattice: the unique stencil on these five
    # neighbours is the 5-point Laplacian (1 on E, N, W, S; 0 on NE)
    off = [(1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1)]
    x = np.array([0.0] + [a for a, _ in off])
    y = np.array([0.0] + [b for _, b in off])
    slots = np.full(32, -1)
    slots[:8] = np.arange(1, 9)
    f0 = np.zeros(32, dtype=np.float32)
    f0[:8] = [0.8, 0.3, 0.9, 0.01, 1.1, 0.02, 0.7, 0.03]
    ok, js, f, fii = mlp.learned_stencil(x, y, 1.0, 0, slots, f0)
    assert ok and js == [1, 3, 5, 7]  # the zero weight on NE is not kept
    assert np.all(f == 1.0) and fii == -4.0


def test_candidates_are_the_small_neighbourhood():
    # a second ring of neighbours carries large proposals but is not in the
    # small neighbourhood: only the eight closest (one per segment) count
    off = [(1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1)]
    x = np.array([0.0] + [a for a, _ in off] + [1.5 * a for a, _ in off])
    y = np.array([0.0] + [b for _, b in off] + [1.5 * b for _, b in off])
    row = list(range(1, 17))
    X, slots = mlp.features(x, y, 1.0, 0, row)
    f0 = np.zeros(32, dtype=np.float32)
    for k in range(16):
        j = slots[k]
        f0[k] = 5.0 if j > 8 else (1.0 if j in (1, 3, 5, 7) else 0.01)
    small = np.arange(1, 9)
    ok, js, f, _ = mlp.learned_stencil(x, y, 1.0, 0, slots, f0, small)
    assert ok and set(js) <= set(range(1, 9))
    assert mlp.support(f0, slots, allowed=small) == sorted(k for k in range(16) if slots[k] <= 8)
