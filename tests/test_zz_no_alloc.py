"""vrm_build_neighbourhoods_noalloc against vrm_build_neighbourhoods.

The no-allocation entry point serves callers that cannot allocate device
memory when they need neighbourhoods (programs that own all device memory in
their own pool, real-time loops with no room for allocator calls).  It keeps
its scratch in one fixed device array shared by every call, so this test makes
calls in a row on different clouds (and the first cloud again) and checks each
against the context-based entry point bit for bit (the outputs are indices and
masks): among them a cloud of exactly the largest size the array holds, and a
wide sparse cloud whose grid needs more cells than the array has, so that the
cell size is doubled.  The file is collected last so that a failure here
leaves every other test already run.
"""
import numpy as np
import pytest

import vrm_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vrm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1508_06379_gb300 as v
    v.build()
    return v


def as_np(nb, n, k_cap):
    cnt = nb["count"].cpu().numpy()[:n]
    idx = nb["idx"].cpu().numpy()[: n * k_cap].reshape(n, k_cap)
    rows = [idx[i, : min(cnt[i], k_cap)].tolist() for i in range(n)]
    return cnt, rows, nb["mask"].cpu().numpy()[:n], nb["small"].cpu().numpy()[: n * 8], nb["max_count"]


def test_noalloc_matches_context_entry_point_twice(vrm):
    clouds = [vrm_inputs.random_cloud(20000, h=0.01, jitter=0.3, seed=1)[:2] + (0.01,),
              vrm_inputs.uniform_scatter(5000, half_width=1.0, seed=3)[:2] + (0.03,)]
    clouds.append(clouds[0])
    # exactly VRM_NOALLOC_MAX_N particles (a 256 x 256 jittered lattice)
    xm, ym = vrm_inputs.random_cloud(vrm.NOALLOC_MAX_N, h=0.01, jitter=0.3, seed=4)[:2]
    assert len(xm) == vrm.NOALLOC_MAX_N
    clouds.append((xm, ym, 0.01))
    # 20,000 particles scattered over [-1, 1]^2 with h = 0.0025: cells of
    # side R h = 0.005 would need 401 x 401 > 2 * 65536 + 1024 cells
    xs, ys = vrm_inputs.uniform_scatter(20000, half_width=1.0, seed=5)[:2]
    assert (np.floor(2.0 / (2 * 0.0025 * (1 + 1e-6))) + 1) ** 2 > 2 * vrm.NOALLOC_MAX_N + 1024
    clouds.append((xs, ys, 0.0025))
    for x, y, h in clouds:
        n = len(x)
        xt = torch.from_numpy(x).cuda()
        yt = torch.from_numpy(y).cuda()
        ctx = vrm.VRM(h=h, nu=1.0)
        ref = as_np(ctx.build_neighbourhoods(xt, yt, n), n, 32)
        got = as_np(vrm.build_neighbourhoods_noalloc(xt, yt, n, h), n, 32)
        assert np.array_equal(ref[0], got[0])
        assert ref[1] == got[1]
        assert np.array_equal(ref[2], got[2])
        assert np.array_equal(ref[3], got[3])
        assert ref[4] == got[4]


def test_noalloc_rejects_clouds_above_its_limit(vrm):
    n = vrm.NOALLOC_MAX_N + 1
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(vrm.VRMError) as ei:
        vrm.build_neighbourhoods_noalloc(x, x, n, 0.01)
    assert ei.value.status == vrm.VRM_ERR_CAPACITY
