"""Training of the weight-proposal network on LP solutions (the learned path).

Data: jittered lattices (jitter amplitude per cloud uniform in [0.1h, 0.4h])
put through the step's own insertion (vrm_insert_reduce with every particle
diffusing), so that the neighbourhoods hold the zero-strength particles the
step inserts at 1.5h, as they do when the network is used; for every
original particle the library builds the neighbourhood of the cloud after
insertion, solves the small-neighbourhood LP (vrm_solve_weights) and, where
it succeeded, stores the input row (vrm_learned_features) and the LP
weights at the slots (vrm_learned_targets).  Training: vrm_mlp_train_step
(tensor-core forward/backward, AdamW) over shuffled batches with a cosine
learning-rate decay.  Everything runs on the GPU through the C ABI; torch
only holds the buffers and draws the batch permutations.
"""
import math
import os

import numpy as np
import torch

from . import binding as B


def cloud(side, h, jitter, seed):
    """A jittered side x side lattice of spacing h centred at 0."""
    rng = np.random.default_rng(seed)
    k = np.arange(side, dtype=np.float64)
    c = (k - 0.5 * (side - 1)) * h
    X, Y = np.meshgrid(c, c, indexing="xy")
    x = X.ravel() + rng.uniform(-jitter * h, jitter * h, X.size)
    y = Y.ravel() + rng.uniform(-jitter * h, jitter * h, Y.size)
    return x, y


def lp_samples(x, y, h, nu=1e-3, device="cuda", insert=True):
    """(X rows, targets) of every original particle of the cloud whose small
    LP succeeded, on the cloud after the step's insertion (insert=True) or
    on the cloud as given."""
    n0 = len(x)
    ctx = B.VRM(h=h, nu=nu)
    cap = 2 * n0 + 1024 if insert else n0
    xb = torch.zeros(cap, dtype=torch.float64, device=device)
    yb = torch.zeros(cap, dtype=torch.float64, device=device)
    xb[:n0] = torch.from_numpy(np.ascontiguousarray(x)).to(device)
    yb[:n0] = torch.from_numpy(np.ascontiguousarray(y)).to(device)
    n = n0
    if insert:
        n, _, _ = ctx.insert_reduce(xb, yb, n0, torch.ones(n0, dtype=torch.float64, device=device))
    xd, yd = xb[:n].contiguous(), yb[:n].contiguous()
    nb = ctx.build_neighbourhoods(xd, yd, n)
    diffused = torch.zeros(n, dtype=torch.uint8, device=device)
    diffused[:n0] = 1
    w = ctx.solve_weights(xd, yd, n, diffused, nb)
    ok = torch.nonzero(w["status"][:n] == B.LP_SMALL).flatten().to(torch.int32)
    m = int(ok.numel())
    X, slots = ctx.learned_features(xd, yd, ok, nb, m)
    T = B.learned_targets(ok, slots, w["cols"], w["f"])
    ctx.close()
    return X[:m], T


def make_dataset(rows, h=1e-3, side=1001, jitter=(0.1, 0.4), seed=1508006, device="cuda"):
    """At least `rows` (input, target) pairs from seeded jittered clouds;
    returns (X bf16 [N_pad, 128], T fp32 [N, 32], N)."""
    rng = np.random.default_rng(seed)
    Xs, Ts, total = [], [], 0
    while total < rows:
        a = float(rng.uniform(*jitter))
        x, y = cloud(side, h, a, int(rng.integers(0, 2 ** 31 - 1)))
        X, T = lp_samples(x, y, h, device=device)
        Xs.append(X)
        Ts.append(T)
        total += int(T.shape[0])
    X = torch.cat(Xs)[:rows]
    T = torch.cat(Ts)[:rows]
    N = int(T.shape[0])
    pad = (N + 127) // 128 * 128
    if pad > N:
        X = torch.cat([X, torch.zeros(pad - N, B.MLP_IN, dtype=torch.bfloat16, device=device)])
    return X.contiguous(), T.contiguous(), N


def init_params(seed=1508007):
    """W ~ N(0, 1/fan_in), b = 0 (float32 vector of MLP_PARAMS)."""
    rng = np.random.default_rng(seed)
    parts = []
    for out, inp in ((256, 96), (256, 256), (256, 256), (32, 256)):
        parts.append(rng.normal(0.0, 1.0 / math.sqrt(inp), out * inp))
        parts.append(np.zeros(out))
    return np.concatenate(parts).astype(np.float32)


def train(X, T, N, epochs=3, batch=4096, lr=1e-3, lr_min=1e-5, weight_decay=0.0, seed=0, net=None, log=None):
    """Trains a network (new unless given) on the N rows of (X, T); returns
    (net, per-step losses)."""
    if net is None:
        net = B.MLP(batch_rows=batch)
        net.set_params(init_params())
    gen = torch.Generator(device="cpu").manual_seed(seed)
    steps_per_epoch = max(1, N // batch)
    total = epochs * steps_per_epoch
    loss = torch.zeros(2, dtype=torch.float32, device=X.device)
    losses = []
    t = 0
    for ep in range(epochs):
        perm = torch.randperm(N, generator=gen).to(torch.int32).to(X.device)
        for k in range(steps_per_epoch):
            t += 1
            cur = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * (t - 1) / max(total - 1, 1)))
            net.train_step(X, T, perm[k * batch:(k + 1) * batch], t, loss_out=loss, lr=cur,
                           weight_decay=weight_decay)
            if k % 50 == 0 or k == steps_per_epoch - 1:
                losses.append((t, float(loss[0])))
                if log:
                    log("epoch %d step %d loss %.5f lr %.2e" % (ep, t, losses[-1][1], cur))
    net.check()
    return net, losses


def cached_network(path=None, rows=2_000_000, epochs=3, log=None, **kw):
    """A trained network, loaded from `path` (float32 .npy of the parameters)
    if present, else trained and saved there."""
    path = path or os.path.join(os.path.expanduser("~"), ".cache", "paper_1508_06379_gb300",
                                "mlp_%d_%d.npy" % (rows, epochs))
    if os.path.exists(path):
        net = B.MLP(batch_rows=kw.get("batch", 4096))
        net.set_params(np.load(path))
        return net, None
    X, T, N = make_dataset(rows)
    net, losses = train(X, T, N, epochs=epochs, net=None, log=log, **kw)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.save(path, net.get_params().cpu().numpy())
    return net, losses
