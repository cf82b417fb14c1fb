"""Certified binary32 pivoting of the small-neighbourhood LPs (schedule field
lp_fp64_pivots = 0, the default) against FP64 pivoting and the FP64 oracle,
through the C ABI.

Every pivot decision of the binary32 run is taken only where the binary32
value is farther from the tolerance than its running error bound; the other
particles are re-run with FP64 pivots.  So both schedules, and the oracle,
give the same stencils bit for bit, and the statistics say how many LPs the
binary32 run handed back (lp_small_rechecked).
"""
import numpy as np
import pytest

import vrm_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = 8


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1508_06379_gb300 as v
    v.build()
    return v


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def cases():
    out = []
    x, y, g = vrm_inputs.random_cloud(20000, h=0.01, jitter=0.3, seed=11)
    out.append(("jitter20k", x, y, g, 0.01, "jittered"))
    x, y, g = vrm_inputs.gaussian_mixture_cloud(h=4e-3, side=181, jitter=0.3, seed=vrm_inputs.SEED_BASE + 2,
                                                half_width=0.36)
    out.append(("mixture181", x, y, g, 4e-3, "jittered"))
    x, y, g = vrm_inputs.uniform_scatter(4000, half_width=1.0, seed=4)
    out.append(("scatter4k", x, y, g, 0.04, "scatter"))
    x, y, g = vrm_inputs.lamb_oseen_lattice(1 / 64, 1.0, 1e-3, 1.0, eps=1e-10)
    out.append(("lattice_h64", x, y, g, 1 / 64, "lattice"))
    return out


CASES = cases()


def solve(lib, ctx, p, fp64):
    from paper_1508_06379_gb300 import autotune
    ctx.set_schedule(dict(autotune.DEFAULT, lp_fp64_pivots=int(fp64)))
    X, Y, D, nb = p["x"], p["y"], p["diffused"], p["nb"]
    n = len(X)
    nbt = dict(count=cu(nb["count"]), idx=cu(nb["idx"].reshape(-1)), small=cu(nb["small"].reshape(-1)))
    w = ctx.solve_weights(cu(X), cu(Y), n, cu(D), nbt)
    return dict(cols=w["cols"].cpu().numpy()[: n * W].reshape(n, W), f=w["f"].cpu().numpy()[: n * W].reshape(n, W),
                fii=w["fii"].cpu().numpy()[:n], status=w["status"].cpu().numpy()[:n], stats=w["stats"])


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_binary32_pivots_match_fp64_and_oracle(lib, orc, case):
    name, x, y, g, h, kind = case
    p = orc.pipeline(x, y, g, h, 1e-3)
    ctx = lib.VRM(h=h, nu=1e-3)
    w32 = solve(lib, ctx, p, fp64=False)
    w64 = solve(lib, ctx, p, fp64=True)
    n = len(p["x"])
    for k in ("cols", "f", "fii", "status"):
        assert np.array_equal(w32[k], w64[k]), k
    wo = p["w"]
    bad = np.nonzero((w32["cols"] != wo["cols"]).any(1) | (w32["f"] != wo["f"]).any(1))[0]
    assert len(bad) == 0, (bad[:5], w32["f"][bad[:5]], wo["f"][bad[:5]])
    assert np.array_equal(w32["fii"], wo["fii"]) and np.array_equal(w32["status"], wo["status"])
    s32, s64 = w32["stats"], w64["stats"]
    # same LPs, same pivot counts: the certified run ends on the FP64 run's bases
    for k in ("lp_small_solved", "lp_small_pivots", "max_pivots", "small_ok", "full_ok", "no_stencil"):
        assert s32[k] == s64[k], (k, s32[k], s64[k])
    assert s64["lp_small_rechecked"] == 0
    solved, rechecked = s32["lp_small_solved"], s32["lp_small_rechecked"]
    assert solved == int(np.sum(p["diffused"][:n])) > 0
    assert 0 <= rechecked <= solved
    if kind == "jittered":
        # most jittered LPs are decided in binary32
        assert rechecked < 0.2 * solved, (rechecked, solved)


def test_binary32_step_matches_oracle_and_counts(lib, orc):
    # one whole vrm_step in the default schedule against the oracle, and the
    # re-run count reported by the step
    x, y, g = vrm_inputs.random_cloud(40000, h=5e-3, jitter=0.3, seed=12)
    h, nu = 5e-3, 1e-3
    dt = (0.5 * h) ** 2 / (4 * nu) / 8
    x2, y2, g2, st_o = orc.step(x, y, g, h, nu, dt)
    n = len(x)
    cap = 2 * n + 1024
    xb = torch.zeros(cap, dtype=torch.float64, device="cuda")
    yb = torch.zeros(cap, dtype=torch.float64, device="cuda")
    xb[:n] = cu(x)
    yb[:n] = cu(y)
    go = torch.zeros(cap, dtype=torch.float64, device="cuda")
    ctx = lib.VRM(h=h, nu=nu)
    assert ctx.get_schedule()["lp_fp64_pivots"] == 0
    n2, st = ctx.step(xb, yb, n, cu(g), go, dt)
    assert n2 == len(x2) and np.array_equal(go.cpu().numpy()[:n2], g2)
    assert 0 < st["lp_small_rechecked"] < 0.2 * st["lp_small_solved"]
