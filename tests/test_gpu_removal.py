"""GPU parity of particle removal (the outlook of Sec. 6.2) against the FP64
oracle, through the C ABI: the removed set, the kept positions and the
redistributed circulations bit-exact (the identity weights come from the
same phase-I rules and the oracle's LU sequence; the gather adds the removed
particles' shares in ascending index)."""
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


def crowded_cloud(n=1600, h=0.02, extra=0.1, seed=3, jitter=0.3):
    x, y, g = vrm_inputs.random_cloud(n, h=h, jitter=jitter, seed=seed)
    rng = np.random.default_rng(seed + 100)
    m = int(extra * len(x))
    k = rng.choice(len(x), m, replace=False)
    x2 = np.concatenate([x, x[k] + rng.uniform(-0.3, 0.3, m) * h])
    y2 = np.concatenate([y, y[k] + rng.uniform(-0.3, 0.3, m) * h])
    g2 = np.concatenate([g, g[k] * rng.uniform(-1, 1, m)])
    return x2, y2, g2, h


def cases():
    out = []
    for seed in (3, 5):
        out.append(("crowded1600_s%d" % seed,) + crowded_cloud(1600, seed=seed))
    out.append(("crowded20k_extra30",) + crowded_cloud(20000, h=0.01, extra=0.3, seed=7))
    x, y, g = vrm_inputs.uniform_scatter(3000, half_width=1.0, seed=2)
    out.append(("scatter3k", x, y, g, 0.04))
    return out


CASES = cases()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_removal_matches_oracle(lib, orc, case):
    name, x, y, g, h = case
    xo, yo, go, removed, cand, _, _ = orc.remove_close(x, y, g, h)
    ctx = lib.VRM(h=h, nu=1e-3)
    X, Y, G, k, st = ctx.remove_close(cu(x), cu(y), cu(g), len(x))
    assert st["remove_candidates"] == cand > 0
    assert k == len(xo) == st["n_out"] and k < len(x)
    assert np.array_equal(X.cpu().numpy(), xo) and np.array_equal(Y.cpu().numpy(), yo)
    Gg = G.cpu().numpy()
    bad = np.nonzero(Gg != go)[0]
    assert len(bad) == 0, (bad[:5], Gg[bad[:5]], go[bad[:5]])
    # a second call on the same context gives the same result
    X2, Y2, G2, k2, _ = ctx.remove_close(cu(x), cu(y), cu(g), len(x))
    assert k2 == k and torch.equal(G2, G) and torch.equal(X2, X)


def test_removal_edge_cases(lib, orc):
    ctx = lib.VRM(h=0.1, nu=1e-3)
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    X, Y, G, k, st = ctx.remove_close(z, z, z, 0)
    assert k == 0
    # a lattice: nothing is closer than r h, nothing changes
    h = 1.0 / 16
    x, y = vrm_inputs.lattice(h, -0.5, 0.5)
    g = np.linspace(1, 2, len(x))
    ctx = lib.VRM(h=h, nu=1e-3)
    X, Y, G, k, st = ctx.remove_close(cu(x), cu(y), cu(g), len(x))
    assert k == len(x) and st["remove_candidates"] == 0
    assert np.array_equal(G.cpu().numpy(), g) and np.array_equal(X.cpu().numpy(), x)
    # coincident pair: the smaller |Gamma| goes, its circulation moves to the ring
    x2, y2, g2 = np.append(x, x[100]), np.append(y, y[100]), np.append(g, 0.5)
    xo, yo, go, removed, cand, _, _ = orc.remove_close(x2, y2, g2, h)
    X, Y, G, k, st = ctx.remove_close(cu(x2), cu(y2), cu(g2), len(x2))
    assert k == len(xo) == len(x) and np.array_equal(G.cpu().numpy(), go)
    # NaN circulation is an argument error
    g3 = g.copy()
    g3[5] = np.nan
    with pytest.raises(lib.VRMError) as e:
        ctx.remove_close(cu(x), cu(y), cu(g3), len(x))
    assert e.value.status == lib.VRM_ERR_ARG
