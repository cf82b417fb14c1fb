"""GPU parity of vrm_step_batched: many independent clouds of uneven size and
spacing advanced by one call (one CUDA graph with one branch per cloud).

Every cloud must come out exactly as the oracle step of that cloud alone
(positions and the diffused set bit-exact, dGamma bit-identical), and as the
single-cloud vrm_step; errors stay confined to the cloud that caused them.
"""
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


def dt_for(h):
    return (0.5 * h) ** 2 / (4 * NU) / 8


def device_cloud(x, y, g, h, cap=None, dt=None):
    n = len(x)
    cap = cap if cap is not None else 2 * n + 1024
    xb = torch.zeros(cap, dtype=torch.float64, device="cuda")
    yb = torch.zeros(cap, dtype=torch.float64, device="cuda")
    xb[:n] = cu(x)
    yb[:n] = cu(y)
    return dict(x=xb, y=yb, gamma_in=cu(g) if n else torch.zeros(1, dtype=torch.float64, device="cuda"),
                gamma_out=torch.zeros(cap, dtype=torch.float64, device="cuda"), n=n, h=h,
                dt=dt if dt is not None else dt_for(h))


def small_batch():
    out = []
    x, y, g = vrm_inputs.random_cloud(900, h=0.05, jitter=0.35, seed=0)
    out.append((x, y, g, 0.05))
    x, y, g = vrm_inputs.random_cloud(20000, h=0.01, jitter=0.3, seed=1)
    out.append((x, y, g, 0.01))
    x, y, g = vrm_inputs.uniform_scatter(3000, half_width=1.0, seed=2)
    out.append((x, y, g, 0.04))
    out.append((np.zeros(0), np.zeros(0), np.zeros(0), 0.03))  # an empty cloud
    x, y, g = vrm_inputs.lamb_oseen_lattice(0.02, 1.0, NU, 1.0, eps=1e-10)
    out.append((x, y, g, 0.02))
    x, y, g = vrm_inputs.gaussian_mixture_cloud(h=3e-3, side=90, jitter=0.3, seed=7, half_width=0.135)
    out.append((x, y, g, 3e-3))
    return out


def check_against_oracle(orc, cloud, dev, n_out, status):
    x, y, g, h = cloud
    assert status == 0
    if len(x) == 0:
        assert n_out == 0
        return
    x2, y2, g2, _ = orc.step(x, y, g, h, NU, dev["dt"])
    assert n_out == len(x2)
    assert np.array_equal(dev["x"][:n_out].cpu().numpy(), x2)
    assert np.array_equal(dev["y"][:n_out].cpu().numpy(), y2)
    got = dev["gamma_out"][:n_out].cpu().numpy()
    assert np.array_equal(got, g2), int(np.count_nonzero(got != g2))


def test_batched_small_clouds_match_oracle(lib, orc):
    batch = small_batch()
    b = lib.VRMBatch(max_clouds=8, nu=NU)
    devs = [device_cloud(*c) for c in batch]
    res, st = b.step(devs)
    for c, d, (n_out, status) in zip(batch, devs, res):
        check_against_oracle(orc, c, d, n_out, status)
    assert st["n_in"] == sum(len(c[0]) for c in batch)
    # a replay of the captured graph with new step sizes (n and dt travel as
    # parameters): compare with single-cloud vrm_step
    for d in devs:
        d["dt"] *= 2.0
        d["gamma_out"].zero_()
    res2, _ = b.step(devs)
    for c, d, (n_out, status) in zip(batch, devs, res2):
        assert status == 0
        x, y, g, h = c
        if len(x) == 0:
            continue
        one = device_cloud(x, y, g, h, cap=d["x"].numel(), dt=d["dt"])
        ctx = lib.VRM(h=h, nu=NU)
        n1, _ = ctx.step(one["x"], one["y"], one["n"], one["gamma_in"], one["gamma_out"], one["dt"])
        assert n1 == n_out
        assert torch.equal(one["x"][:n1], d["x"][:n1]) and torch.equal(one["gamma_out"][:n1], d["gamma_out"][:n1])


def test_batched_subset_and_changed_spacing(lib, orc):
    # fewer clouds than slots, then a changed spacing: the graph is recaptured
    batch = small_batch()[:3]
    b = lib.VRMBatch(max_clouds=8, nu=NU)
    devs = [device_cloud(*c) for c in batch]
    res, _ = b.step(devs)
    for c, d, (n_out, status) in zip(batch, devs, res):
        check_against_oracle(orc, c, d, n_out, status)
    x, y, g, _ = batch[1]
    batch[1] = (x, y, g, 0.011)
    devs[1] = device_cloud(*batch[1])
    res, _ = b.step(devs[:2])
    for c, d, (n_out, status) in zip(batch[:2], devs[:2], res):
        check_against_oracle(orc, c, d, n_out, status)


def test_batched_errors_stay_in_their_cloud(lib, orc):
    v = lib
    batch = small_batch()[:3]
    b = v.VRMBatch(max_clouds=4, nu=NU)
    devs = [device_cloud(*c) for c in batch]
    # cloud 0: capacity too small for its insertions
    x, y, g, h = batch[0]
    devs[0] = device_cloud(x, y, g, h, cap=len(x) + 2)
    # cloud 2: a NaN circulation
    g_nan = batch[2][2].copy()
    g_nan[7] = np.nan
    devs[2] = device_cloud(batch[2][0], batch[2][1], g_nan, batch[2][3])
    res, _ = b.step(devs, raise_on_error=False)
    assert res[0][1] == v.VRM_ERR_CAPACITY
    x2, _, _, _ = orc.step(x, y, g, h, NU, devs[0]["dt"])
    # the count after the round that did not fit: above the capacity, at most the final count
    assert len(x) + 2 < res[0][0] <= len(x2)
    assert res[2][1] == v.VRM_ERR_ARG
    check_against_oracle(orc, batch[1], devs[1], *res[1])
    with pytest.raises(v.VRMError):
        b.step(devs)
    # the batch stays usable
    devs = [device_cloud(*c) for c in batch]
    res, _ = b.step(devs)
    for c, d, (n_out, status) in zip(batch, devs, res):
        check_against_oracle(orc, c, d, n_out, status)


def test_batched_graph_and_eager_agree(lib, monkeypatch):
    batch = small_batch()
    outs = []
    for env in ("0", "1"):
        monkeypatch.setenv("VRM_NO_GRAPH", env)
        b = lib.VRMBatch(max_clouds=8, nu=NU)
        devs = [device_cloud(*c) for c in batch]
        res, st = b.step(devs)
        outs.append([(r[0], d["x"][:r[0]].cpu(), d["gamma_out"][:r[0]].cpu()) for r, d in zip(res, devs)])
    for a, c in zip(outs[0], outs[1]):
        assert a[0] == c[0] and torch.equal(a[1], c[1]) and torch.equal(a[2], c[2])


@pytest.mark.slow
def test_batched_64_clouds_full_size(lib, orc):
    # the 64-cloud workload that bench.py times (log-uniform 1e4..5e5
    # particles, h ~ U[1e-3, 4e-3]) in the same launch configuration: every
    # cloud against the single-cloud vrm_step, every eighth against the oracle
    clouds = vrm_inputs.batched_clouds()
    b = lib.VRMBatch(max_clouds=len(clouds), nu=NU)
    devs = [device_cloud(x, y, g, h, cap=int(1.6 * len(x)) + 4096) for x, y, g, h in clouds]
    res, st = b.step(devs)
    assert all(r[1] == 0 for r in res)
    assert st["n_in"] == sum(len(c[0]) for c in clouds)
    ctx_by_h = {}
    for k, (c, d, (n_out, status)) in enumerate(zip(clouds, devs, res)):
        x, y, g, h = c
        if k % 8 == 0:
            check_against_oracle(orc, c, d, n_out, status)
        one = device_cloud(x, y, g, h, cap=d["x"].numel(), dt=d["dt"])
        ctx = ctx_by_h.setdefault(h, lib.VRM(h=h, nu=NU))
        n1, _ = ctx.step(one["x"], one["y"], one["n"], one["gamma_in"], one["gamma_out"], one["dt"])
        assert n1 == n_out
        assert torch.equal(one["x"][:n1], d["x"][:n1]) and torch.equal(one["gamma_out"][:n1], d["gamma_out"][:n1])
