"""A few VRM diffusion steps on a jittered-lattice Gaussian-mixture cloud of a
chosen lattice side, for kernel profilers (ncu) and quick timing.

    VRM_NO_GRAPH=1 python -m paper_1508_06379_gb300.profile_step --side 701 --steps 2 --lp-block 384

The cloud is the 1M-particle workload's recipe (h = 2e-3, jitter 0.3 h,
eight Gaussians) on a side x side lattice; --side 1001 is the full workload.
VRM_NO_GRAPH=1 runs the step's kernels eagerly (profilers that do not profile
kernel nodes inside conditional graph nodes see every launch that way).
Prints the particle counts of the last step.
"""
import argparse
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--side", type=int, default=701, help="lattice side (1001: the 1M-particle cloud)")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--lp-block", type=int, default=384,
                    help="schedule lp_block (384 / 192: warp-specialised binary32 LP; 32..128: one LP per thread)")
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch
    import vrm_inputs
    import paper_1508_06379_gb300 as vrm
    from paper_1508_06379_gb300 import autotune

    h, nu = 2e-3, 1e-3
    x, y, g = vrm_inputs.gaussian_mixture_cloud(h=h, side=a.side, jitter=0.3, seed=vrm_inputs.SEED_BASE + 2,
                                                half_width=0.5 * (a.side - 1) * h)
    dt = (0.5 * h) ** 2 / (4 * nu) / 8
    n = len(x)
    cap = int(n * 1.6) + 4096
    xb = torch.zeros(cap, dtype=torch.float64, device="cuda")
    yb = torch.zeros_like(xb)
    xb[:n] = torch.from_numpy(x).cuda()
    yb[:n] = torch.from_numpy(y).cuda()
    gi = torch.from_numpy(g).cuda()
    go = torch.zeros_like(xb)
    ctx = vrm.VRM(h=h, nu=nu)
    per_sm = {384: 1, 192: 2}.get(a.lp_block, autotune.DEFAULT["lp_blocks_per_sm"])
    ctx.set_schedule(dict(autotune.DEFAULT, lp_block=a.lp_block, lp_blocks_per_sm=per_sm))
    n2, st = n, {}
    for _ in range(a.steps):
        n2, st = ctx.step(xb, yb, n, gi, go, dt)
    torch.cuda.synchronize()
    print("n %d n_out %d n_diffused %d lp_small_rechecked %d" % (n, n2, st["n_diffused"], st["lp_small_rechecked"]))


if __name__ == "__main__":
    main()
