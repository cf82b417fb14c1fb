"""The weight-proposal network on the tensor cores against the FP64 oracle
(oracle/mlp.py): forward pass, gradients and AdamW, all through the C ABI.

Tolerances.  The GPU keeps weights and activations in bf16 (8 significant
bits, unit roundoff u = 2^-9) and accumulates in fp32.  The oracle is run on
the same bf16 weights and inputs with its hidden activations rounded to bf16
as well, so the two differ only by fp32 accumulation order and by
activations whose bf16 rounding falls differently (one bf16 ulp, 2^-8
relative); over 256-term sums of O(1) terms that stays below 1e-2 of the
output scale.  Gradients carry the same effect plus bf16 rounding of the
back-propagated errors: the bar is a relative Frobenius error of 2e-2 per
parameter block.  AdamW runs in fp32 against the oracle's FP64: 2e-6.
"""
import numpy as np
import pytest

import vrm_inputs
from oracle import mlp as omlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1508_06379_gb300 as v
    v.build()
    return v


def quantised(theta):
    """The parameters as the GPU uses them: bf16 weights, fp32 biases."""
    out = theta.astype(np.float32).astype(np.float64)
    o = 0
    for rows, cols in omlp.SHAPES:
        out[o:o + rows * cols] = omlp.to_bf16(theta[o:o + rows * cols])
        o += rows * cols + rows
    return out


def term_scale(theta, cache, dY):
    """Per gradient entry, the sum of the magnitudes of the products that
    make it up: the backward pass of the oracle's network with every factor
    (output gradient, GELU derivative, weight, activation) replaced by its
    absolute value."""
    layers = omlp.unflatten(theta)
    grads = [None] * len(layers)
    g = np.abs(dY)
    for l in range(len(layers) - 1, -1, -1):
        a, z = cache[l]
        if l < len(layers) - 1:
            g = g * np.abs(omlp.gelu_grad(z))
        W, _ = layers[l]
        grads[l] = (g.T @ np.abs(a), g.sum(axis=0))
        g = g @ np.abs(W)
    return omlp.flatten(grads)


def bf16_rows(X):
    return torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).cuda()


def blocks(v):
    out, o = [], 0
    for rows, cols in omlp.SHAPES:
        out.append(v[o:o + rows * cols])
        o += rows * cols
        out.append(v[o:o + rows])
        o += rows
    return out


# 40,000 and 60,000 rows: 313 and 469 tiles, so that the persistent CTAs
# (one per SM) take two to four tiles each, whole pairs and a last single one
@pytest.mark.parametrize("rows", [128, 1000, 4096, 40000, 60000])
def test_forward_matches_oracle(lib, rows):
    theta = vrm_inputs.mlp_params()
    X, _ = vrm_inputs.mlp_rows(rows, seed=11)
    net = lib.MLP(batch_rows=128)
    net.set_params(theta)
    Y = net.forward(bf16_rows(X)).cpu().numpy().astype(np.float64)
    Yo, _ = omlp.forward(quantised(theta), X[:, :96], bf16_acts=True)
    scale = max(1.0, float(np.max(np.abs(Yo))))
    err = np.abs(Y - Yo)
    assert np.max(err) <= 1e-2 * scale, np.max(err)
    assert np.mean(err) <= 1e-3 * scale, np.mean(err)
    # against the unrounded FP64 network: the bf16 path's own error, stated
    Yf, _ = omlp.forward(quantised(theta), X[:, :96], bf16_acts=False)
    assert np.max(np.abs(Y - Yf)) <= 5e-2 * scale


@pytest.mark.parametrize("B,rows", [(128, 128), (512, 512), (512, 300)])
def test_gradients_match_oracle(lib, B, rows):
    theta = vrm_inputs.mlp_params()
    X, T = vrm_inputs.mlp_rows(rows, seed=12)
    net = lib.MLP(batch_rows=B)
    net.set_params(theta)
    g, loss = net.grads(bf16_rows(X), torch.from_numpy(T.astype(np.float32)).cuda())
    g = g.cpu().numpy().astype(np.float64)
    thq = quantised(theta)
    Yo, cache = omlp.forward(thq, X[:, :96], bf16_acts=True)
    lo, dY = omlp.loss(Yo, T, X[:, 64:96])
    go = omlp.backward(thq, cache, dY)
    assert abs(loss - lo) <= 2e-2 * lo
    for k, (a, b) in enumerate(zip(blocks(g), blocks(go))):
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        cos = float(a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))
        assert rel <= 2e-2 and cos >= 0.999, (k, rel, cos)
    # element by element: each gradient entry is a sum of products (rows x
    # backpropagated terms); its error may be a bf16-sized fraction of the
    # sum of those products' magnitudes, not more
    sc = term_scale(thq, cache, dY)
    for k, (a, b, s) in enumerate(zip(blocks(g), blocks(go), blocks(sc))):
        excess = np.abs(a - b) - (2e-2 * s + 1e-30)
        worst = int(np.argmax(excess))
        assert excess[worst] <= 0, (k, worst, a[worst], b[worst], s[worst])
    # the padded input columns of W1 receive no gradient (they are not parameters)
    assert np.all(np.isfinite(g))


def test_adamw_matches_oracle(lib):
    theta = vrm_inputs.mlp_params()
    net = lib.MLP(batch_rows=128)
    net.set_params(theta)
    hp = dict(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.01)
    th = theta.astype(np.float32).astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    for t in (1, 2, 3):
        g = vrm_inputs.mlp_vector(100 + t, scale=0.1)
        net.adamw(torch.from_numpy(g.astype(np.float32)).cuda(), t, **hp)
        th, m, v = omlp.adamw(th, g.astype(np.float32).astype(np.float64), m, v, t, **hp)
    got = net.get_params().cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - th)) <= 2e-6


def test_training_is_deterministic_and_lowers_the_loss(lib):
    X, T = vrm_inputs.mlp_rows(4096, seed=13)
    Xd = bf16_rows(X)
    Td = torch.from_numpy(T.astype(np.float32)).cuda()
    runs = []
    for _ in range(2):
        net = lib.MLP(batch_rows=512)
        net.set_params(vrm_inputs.mlp_params())
        loss = torch.zeros(2, dtype=torch.float32, device="cuda")
        losses = []
        gen = torch.Generator(device="cpu").manual_seed(0)
        for t in range(1, 121):
            idx = torch.randperm(4096, generator=gen)[:512].to(torch.int32).cuda()
            net.train_step(Xd, Td, idx, t, loss_out=loss, lr=1e-3)
            losses.append(float(loss[0]))
        net.check()
        runs.append((losses, net.get_params().cpu()))
    assert runs[0][0] == runs[1][0] and torch.equal(runs[0][1], runs[1][1])
    losses = runs[0][0]
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:10])
