"""Launch schedules (vrm_schedule) and their autotuner on the GPU: every
schedule gives the same bits, a row_cap that cuts rows is repeated with whole
rows, and the tuned schedules are cached and applied to batches."""
import numpy as np
import pytest

import vrm_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NU = 1e-3


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1508_06379_gb300 as v
    v.build()
    return v


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def device_cloud(x, y, g, h, cap=None):
    n = len(x)
    cap = cap or 2 * n + 1024
    xb = torch.zeros(cap, dtype=torch.float64, device="cuda")
    yb = torch.zeros(cap, dtype=torch.float64, device="cuda")
    xb[:n] = cu(x)
    yb[:n] = cu(y)
    return dict(x=xb, y=yb, gamma_in=cu(g), gamma_out=torch.zeros(cap, dtype=torch.float64, device="cuda"), n=n,
                h=h, dt=(0.5 * h) ** 2 / (4 * NU) / 8)


def run(ctx, d):
    n2, st = ctx.step(d["x"], d["y"], d["n"], d["gamma_in"], d["gamma_out"], d["dt"])
    return n2, d["x"][:n2].clone(), d["gamma_out"][:n2].clone(), st


def test_every_schedule_gives_the_same_bits(lib, orc):
    from paper_1508_06379_gb300 import autotune
    x, y, g = vrm_inputs.random_cloud(20000, h=0.01, jitter=0.3, seed=1)
    d = device_cloud(x, y, g, 0.01)
    ctx = lib.VRM(h=0.01, nu=NU)
    n2, x2, g2, st = run(ctx, d)
    x_o, _, g_o, _ = orc.step(x, y, g, 0.01, NU, d["dt"])
    assert np.array_equal(g2.cpu().numpy(), g_o)
    for _, options in autotune.GROUPS:
        for opt in options:
            s = dict(autotune.DEFAULT, **opt)
            if s["row_cap"] < st["max_count"]:
                continue
            ctx.set_schedule(s)
            m, xs, gs, _ = run(ctx, d)
            assert m == n2 and torch.equal(xs, x2) and torch.equal(gs, g2), s
            assert ctx.get_schedule() == s


def test_cut_rows_are_repeated_with_whole_rows(lib):
    x, y, g = vrm_inputs.gaussian_mixture_cloud(h=3e-3, side=90, jitter=0.3, seed=7, half_width=0.135)
    d = device_cloud(x, y, g, 3e-3)
    ctx = lib.VRM(h=3e-3, nu=NU)
    n2, x2, g2, st = run(ctx, d)
    assert st["max_count"] > 16  # the mixture cloud has rows wider than 16
    from paper_1508_06379_gb300 import autotune
    ctx.set_schedule(dict(autotune.DEFAULT, row_cap=16))
    m, xs, gs, st2 = run(ctx, d)
    assert m == n2 and torch.equal(xs, x2) and torch.equal(gs, g2)
    assert ctx.get_schedule()["row_cap"] == 32 and st2["max_count"] == st["max_count"]
    # the same in a batch
    b = lib.VRMBatch(max_clouds=2, nu=NU)
    b.set_schedule(0, dict(autotune.DEFAULT, row_cap=16))
    d2 = device_cloud(x, y, g, 3e-3)
    res, _ = b.step([d2])
    assert res[0] == (n2, 0)
    assert torch.equal(d2["x"][:n2], x2) and torch.equal(d2["gamma_out"][:n2], g2)


def test_invalid_schedules_are_argument_errors(lib):
    from paper_1508_06379_gb300 import autotune
    ctx = lib.VRM(h=0.01, nu=NU)
    for bad in (dict(row_cap=40), dict(row_cap=4), dict(search_block=48), dict(search_block=512),
                dict(lp_block=256), dict(lp_blocks_per_sm=0), dict(apply_block=0)):
        with pytest.raises(lib.VRMError) as ei:
            ctx.set_schedule(dict(autotune.DEFAULT, **bad))
        assert ei.value.status == lib.VRM_ERR_ARG
    b = lib.VRMBatch(max_clouds=2, nu=NU)
    with pytest.raises(lib.VRMError):
        b.set_schedule(2, autotune.DEFAULT)


def test_autotuner_tunes_caches_and_applies(lib, tmp_path):
    from paper_1508_06379_gb300 import autotune
    path = str(tmp_path / "schedules.json")
    x, y, g = vrm_inputs.random_cloud(20000, h=0.01, jitter=0.3, seed=1)
    d = device_cloud(x, y, g, 0.01)
    ref = lib.VRM(h=0.01, nu=NU)
    n2, x2, g2, _ = run(ref, device_cloud(x, y, g, 0.01))
    tuner = autotune.Autotuner(path, reps=2)
    ctx = lib.VRM(h=0.01, nu=NU)
    s = tuner.apply(ctx, d)
    assert ctx.get_schedule() == s
    assert autotune.Autotuner(path).lookup(32, 20000) == s
    m, xs, gs, _ = run(ctx, d)
    assert m == n2 and torch.equal(xs, x2) and torch.equal(gs, g2)
    # a batch of clouds in two buckets gets one schedule per bucket
    clouds = [(x, y, g, 0.01)]
    xb_, yb_, gb_ = vrm_inputs.random_cloud(2000, h=0.05, jitter=0.3, seed=5)
    clouds.append((xb_, yb_, gb_, 0.05))
    devs = [device_cloud(*c) for c in clouds]
    b = lib.VRMBatch(max_clouds=4, nu=NU)
    chosen = tuner.tune_batch(b, devs)
    assert set(chosen) == {0, 1} and chosen[0] == s
    res, _ = b.step(devs)
    assert res[0] == (n2, 0)
    assert torch.equal(devs[0]["x"][:n2], x2) and torch.equal(devs[0]["gamma_out"][:n2], g2)
    one = lib.VRM(h=0.05, nu=NU)
    m1, x1, g1, _ = run(one, device_cloud(*clouds[1]))
    assert res[1] == (m1, 0) and torch.equal(devs[1]["gamma_out"][:m1], g1)
