#!/usr/bin/env python3
"""Throughput of one VRM diffusion step (vrm_step) on one GB300.

Workload (default): the 1,002,001-particle lattice of spacing h = 2e-3 on
[-1, 1]^2, jittered by U(-0.3h, 0.3h) per coordinate (seed 1508002), carrying
a mixture of 8 Gaussian vortices; nu = 1e-3, growth control (C_diff = 1) and
insertion on, Euler step dt = (1/8)(r h)^2/(4 nu).  A step is the whole
operator: growth control, insertion rounds, neighbourhoods, LP weights,
application and Euler update.  Metric: particles per second, counted after
insertion (n'), whole job.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the launching stream with an L2 flush (a 512 MB write) between steps,
outside the events.  Every step takes the same input (the step is
idempotent: it reads gamma_in and writes gamma_out and the appended
positions), so every step does the same work.

--impl reference times the CPU oracle (oracle/, FP64 C with OpenMP) on a
bounded sample of the same workload with the same metric.
Under torchrun (N > 1) every rank runs its own replica (replicas only: the
operator is evaluated on one GPU per cloud, with no collective on the data
path); the value is the sum of particles over ranks / the slowest rank's time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particles/s per VRM diffusion step on 1 GB300; learned vs plain LP at equal error"
UNIT = "particles/s"
# derived FP64 peak, shown beside the measured one: 152 SMs x 2 FP64 FMA
# lanes/clk x 2 flop x 2.07 GHz (GFLOP/s)
FP64_PEAK_DERIVED_GFLOPS = 152 * 2 * 2 * 2.07


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mixture_1m",
                    choices=["mixture_1m", "mixture_1m_n2", "lamb_oseen_h002", "batched_64", "learned_4m",
                             "viscous_16m", "removal_1m"])
    ap.add_argument("--learned", action="store_true",
                    help="viscous workload: stencils from a trained proposal network (LP fallback)")
    ap.add_argument("--viscous-h", type=float, default=7 * 2.0 ** -16,
                    help="lattice spacing of the viscous Lamb-Oseen workload (7 2^-16 = 1.068e-4: about 15.5M "
                         "particles, binary-exact lattice coordinates)")
    ap.add_argument("--train-rows", type=int, default=10_000_000,
                    help="LP solutions the network of the learned workload is trained on")
    ap.add_argument("--train-epochs", type=int, default=3)
    ap.add_argument("--learned-side", type=int, default=2001,
                    help="lattice side of the learned workload's cloud (2001: the 4M-particle cloud)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true",
                    help="default workload: skip the learned-vs-LP comparison block")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch schedule")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="mixed: the application accumulates in fp32 (dGamma within 1e-5 of the term scale)")
    ap.add_argument("--schedule-cache", default=None,
                    help="JSON cache of tuned schedules (default: $VRM_SCHEDULE_CACHE or ~/.cache)")
    return ap.parse_args()


def workload(name, rank=0):
    import vrm_inputs
    if name in ("mixture_1m", "mixture_1m_n2"):
        h, nu = 2e-3, 1e-3
        x, y, g = vrm_inputs.gaussian_mixture_cloud(h=h, jitter=0.3, seed=vrm_inputs.SEED_BASE + 2 + 1000 * rank)
        desc = {"workload": "jittered lattice 1001x1001, h=2e-3, jitter 0.3h, 8-Gaussian mixture, nu=1e-3, "
                            "C_diff=1, insertion on, FP64", "n": int(len(x)), "h": h, "nu": nu, "order": 1, "R": 2.0}
        if name == "mixture_1m_n2":
            # n = 2: nine moment rows; R = 2.5 because with R = 2 about a
            # third of the jittered particles have no non-negative stencil
            desc.update(order=2, R=2.5)
            desc["workload"] = desc["workload"].replace("FP64", "n=2 (cubic moments), R=2.5, FP64")
    else:
        h, nu = 0.02, 1e-3
        x, y, g = vrm_inputs.lamb_oseen_lattice(h, 1.0, nu, 1.0, eps=1e-10)
        desc = {"workload": "Lamb-Oseen lattice h=0.02, Gamma=1, nu=1e-3, t0=1, |omega|>1e-10", "n": int(len(x)),
                "h": h, "nu": nu, "order": 1, "R": 2.0}
    dt = (0.5 * h) ** 2 / (4 * nu) / 8
    desc["dt"] = dt
    return x, y, g, h, nu, dt, desc


def sample_window(x, y, g, frac):
    """Centred square window holding about `frac` of the cloud."""
    import numpy as np
    lo_x, hi_x = x.min(), x.max()
    lo_y, hi_y = y.min(), y.max()
    a = 0.5 * math.sqrt(frac)
    cx, cy = 0.5 * (lo_x + hi_x), 0.5 * (lo_y + hi_y)
    keep = (np.abs(x - cx) <= a * (hi_x - lo_x)) & (np.abs(y - cy) <= a * (hi_y - lo_y))
    return x[keep].copy(), y[keep].copy(), g[keep].copy()


class Clocks:
    """SM clock, power and clock-event reasons sampled while the timed region
    runs: read-only NVML queries (libnvidia-ml through ctypes) every 5 ms from
    a thread, else nvidia-smi queries every 200 ms."""

    # clock event reason bits (nvml.h): hw slowdown, sw thermal, hw thermal, sw power cap
    REASONS = {0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown", 0x4: "sw_power_cap"}

    def __init__(self, gpu_uuid=None):
        self.samples = []  # (t, sm_mhz, max_mhz, power_w, reasons bitmask or names)
        self.stop_flag = False
        self.nvml = None
        self.handle = None
        try:
            import ctypes
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() == 0:
                h = ctypes.c_void_p()
                ok = -1
                if gpu_uuid:
                    ok = lib.nvmlDeviceGetHandleByUUID(gpu_uuid.encode(), ctypes.byref(h))
                if ok != 0:
                    ok = lib.nvmlDeviceGetHandleByIndex_v2(0, ctypes.byref(h))
                if ok == 0:
                    self.nvml, self.handle, self.ct = lib, h, ctypes
                    self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                        getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons", None)
        except Exception:
            self.nvml = None
        self.cmd = ["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
                    "clocks_event_reasons.hw_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                    "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                    "--format=csv,noheader,nounits"]
        if gpu_uuid:
            self.cmd += ["-i", gpu_uuid]
        self.thread = threading.Thread(target=self._poll, daemon=True)
        self.thread.start()

    def _nvml_sample(self):
        ct, lib, h = self.ct, self.nvml, self.handle
        clk, mx, pw, rs = ct.c_uint(), ct.c_uint(), ct.c_uint(), ct.c_ulonglong()
        lib.nvmlDeviceGetClockInfo(h, 1, ct.byref(clk))  # NVML_CLOCK_SM
        lib.nvmlDeviceGetMaxClockInfo(h, 1, ct.byref(mx))
        lib.nvmlDeviceGetPowerUsage(h, ct.byref(pw))
        names = []
        if self.reasons_fn is not None and self.reasons_fn(h, ct.byref(rs)) == 0:
            names = [n for bit, n in self.REASONS.items() if rs.value & bit]
        return (time.time(), float(clk.value), float(mx.value), pw.value / 1000.0, names)

    def _poll(self):
        while not self.stop_flag:
            t = time.time()
            try:
                if self.nvml is not None:
                    self.samples.append(self._nvml_sample())
                    time.sleep(0.005)
                    continue
                out = subprocess.run(self.cmd, capture_output=True, text=True, timeout=5).stdout
                for line in out.splitlines():
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) < 7:
                        continue
                    names = [n for n, v in zip(["hw_slowdown", "sw_thermal_slowdown", "hw_thermal_slowdown",
                                                "sw_power_cap"], parts[3:7]) if v.lower() == "active"]
                    self.samples.append((t, float(parts[0]), float(parts[1]), float(parts[2]), names))
            except Exception:
                pass
            time.sleep(max(0.0, 0.2 - (time.time() - t)))

    def stop(self, t0, t1):
        self.stop_flag = True
        self.thread.join(timeout=10)
        sel = [s for s in self.samples if t0 <= s[0] <= t1]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no clock samples"], "samples": 0}
        reasons = sorted({n for s in sel for n in s[4]})
        return {"sm_mhz": statistics.median(s[1] for s in sel), "sm_max_mhz": max(s[2] for s in sel),
                "reasons": reasons, "samples": len(sel), "power_w_max": max(s[3] for s in sel),
                "source": "nvml" if self.nvml is not None else "nvidia-smi"}


def lp_flops(n_lp, pivots, m=5, K=8, cols=None, col_pivots=None):
    """Algorithmic FP64 flops of phase-I LPs with m rows on K columns (a
    multiply-add counts 2): per LP, per column 2 offsets + 3 distance + 2
    scalings + (m - 2) Vandermonde products + m cost-row sums, then the final
    residual (m K multiply-adds, m differences) and f~_ii (K sums); per pivot
    m ratio divisions, K + 1 pivot-row scalings and the (m + 1)(K + 1)
    multiply-adds of the tableau update.  m = 5, K = 8: 213 per LP and 122 per
    pivot.  For the full-neighbourhood LPs K varies: `cols` = sum of K and
    `col_pivots` = sum of K x pivots over the LPs."""
    if cols is None:
        cols, col_pivots = n_lp * K, pivots * K
    per_col = 7 + (m - 2) + m + 2 * m + 1
    return cols * per_col + n_lp * m + pivots * (m + 1 + 2 * (m + 1)) + col_pivots * (1 + 2 * (m + 1))


def lp_flops_certified(n_lp, n_rechecked, pivots, K=8):
    """FP64 flops of the small LPs with certified binary32 pivots (n = 1):
    per LP the column setup (7 per column) and the FP64 solve of the final
    basis (5 x 5 LU 75, substitutions 45, basis columns 15, sums 12: 147;
    the residual is certified by the LU backward error and not computed),
    and for the LPs re-run with FP64 pivots their whole FP64 LP (lp_flops,
    at the mean pivot count)."""
    mean_piv = pivots / max(n_lp, 1)
    return n_lp * (7 * K + 147) + lp_flops(n_rechecked, n_rechecked * mean_piv, 5, K)


def run_ours(args):
    import numpy as np
    import torch

    import paper_1508_06379_gb300 as vrm

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    vrm.build()
    x, y, g, h, nu, dt, desc = workload(args.workload, rank)
    n = len(x)
    cap = int(n * 1.6) + 4096
    dev = torch.device("cuda", local)
    xb = torch.zeros(cap, dtype=torch.float64, device=dev)
    yb = torch.zeros(cap, dtype=torch.float64, device=dev)
    xb[:n] = torch.from_numpy(x).to(dev)
    yb[:n] = torch.from_numpy(y).to(dev)
    gi = torch.from_numpy(g).to(dev)
    go = torch.zeros(cap, dtype=torch.float64, device=dev)
    ctx = vrm.VRM(h=h, nu=nu, precision=args.precision, order=desc["order"], R=desc["R"])
    schedule = None
    if not args.no_autotune:
        from paper_1508_06379_gb300 import autotune
        schedule = autotune.Autotuner(args.schedule_cache).apply(
            ctx, dict(x=xb, y=yb, n=n, gamma_in=gi, gamma_out=go, dt=dt))
    ctx.set_timing(True)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        flush.zero_()
        ctx.step(xb, yb, n, gi, go, dt)
    torch.cuda.synchronize()
    # the FP64/FP32 FMA rate of this GPU (k_fma_probe): the LP's roofline
    # denominator, measured in this run
    peaks = {"fp64_tflops": vrm.fma_peak(True) / 1e12, "fp32_tflops": vrm.fma_peak(False) / 1e12}
    gpu_id = None
    try:
        gpu_id = str(torch.cuda.get_device_properties(local).uuid)
        gpu_id = gpu_id if gpu_id.startswith("GPU-") else "GPU-" + gpu_id
    except Exception:
        gpu_id = None
    clocks = Clocks(gpu_id)
    time.sleep(0.5)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = vrm.launch_count()
    t_wall0 = time.time()
    total_ms = 0.0
    parts = 0
    stage_ms = {k: [] for k in vrm.STAGES}
    stats = None
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n2, stats = ctx.step(xb, yb, n, gi, go, dt)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        parts += n2
        try:
            for k, v in ctx.stage_times().items():
                stage_ms[k].append(v)
        except Exception:
            pass
    torch.cuda.synchronize()
    t_wall1 = time.time()
    launches = vrm.launch_count() - launches0
    ck = clocks.stop(t_wall0, t_wall1)
    if dist:
        t = torch.tensor([total_ms, float(parts)], dtype=torch.float64, device=dev)
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        total_ms_max, parts_all = tmax[0].item(), t[1].item()
    else:
        total_ms_max, parts_all = total_ms, float(parts)
    value = parts_all / (total_ms_max * 1e-3)

    # end to end through the C ABI with host buffers: h2d of the inputs and d2h
    # of the result (gamma_out and appended positions) inside the timed region
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.from_numpy(y).pin_memory()
    gh = torch.from_numpy(g).pin_memory()
    go_h = torch.empty(cap, dtype=torch.float64).pin_memory()
    xo_h = torch.empty(cap, dtype=torch.float64).pin_memory()
    yo_h = torch.empty(cap, dtype=torch.float64).pin_memory()
    h2d = 24 * n
    e2e_steps = max(1, min(args.steps, 5))
    # (a) serial: each step copies in, steps, copies out, with an L2 flush
    # between steps outside the events
    ser_ms, ser_parts = 0.0, 0
    for _ in range(e2e_steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xb[:n].copy_(xh, non_blocking=True)
        yb[:n].copy_(yh, non_blocking=True)
        gi.copy_(gh, non_blocking=True)
        n2, _ = ctx.step(xb, yb, n, gi, go, dt, stats=False)
        go_h[:n2].copy_(go[:n2], non_blocking=True)
        xo_h[n:n2].copy_(xb[n:n2], non_blocking=True)
        yo_h[n:n2].copy_(yb[n:n2], non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        ser_ms += e0.elapsed_time(e1)
        ser_parts += n2
    d2h = 8 * n2 + 16 * (n2 - n)
    # (b) pipelined, as a stream of steps runs: two buffer sets (each with its
    # own context, so each keeps its captured step), the inputs of step k + 1
    # copied in and the results of step k - 1 copied out on a second stream
    # while step k runs; one pair of events around all the steps
    sets = [dict(x=xb, y=yb, gi=gi, go=go, ctx=ctx)]
    ctx2 = vrm.VRM(h=h, nu=nu, precision=args.precision, order=desc["order"], R=desc["R"])
    ctx2.set_schedule(ctx.get_schedule())
    sets.append(dict(x=torch.zeros_like(xb), y=torch.zeros_like(yb), gi=torch.empty_like(gi),
                     go=torch.zeros_like(go), ctx=ctx2))
    cs = torch.cuda.Stream(device=dev)
    ready = [torch.cuda.Event() for _ in sets]

    def copy_in(k):
        b = sets[k % 2]
        with torch.cuda.stream(cs):
            b["x"][:n].copy_(xh, non_blocking=True)
            b["y"][:n].copy_(yh, non_blocking=True)
            b["gi"].copy_(gh, non_blocking=True)
            ready[k % 2].record(cs)

    for k in range(2):  # capture each context's step once, outside the timing
        copy_in(k)
        stream.wait_event(ready[k])
        sets[k]["ctx"].step(sets[k]["x"], sets[k]["y"], n, sets[k]["gi"], sets[k]["go"], dt, stats=False)
    torch.cuda.synchronize()
    flush.zero_()
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    done = [torch.cuda.Event() for _ in sets]

    def begin(k):
        b = sets[k % 2]
        stream.wait_event(ready[k % 2])
        # L2 flushed before every step (inside the timed region here): the
        # step starts cold, as in the device-side measurement
        flush.zero_()
        b["ctx"].step_begin(b["x"], b["y"], n, b["gi"], b["go"], dt)
        done[k % 2].record(stream)

    p0.record(cs)
    copy_in(0)
    begin(0)
    pipe_parts = 0
    for k in range(args.steps):
        # step k + 1 is queued behind step k before step k is waited for
        if k + 1 < args.steps:
            copy_in(k + 1)
            begin(k + 1)
        b = sets[k % 2]
        n2, _ = b["ctx"].step_end(stats=False)
        pipe_parts += n2
        with torch.cuda.stream(cs):
            cs.wait_event(done[k % 2])
            go_h[:n2].copy_(b["go"][:n2], non_blocking=True)
            xo_h[n:n2].copy_(b["x"][n:n2], non_blocking=True)
            yo_h[n:n2].copy_(b["y"][n:n2], non_blocking=True)
    p1.record(cs)
    p1.synchronize()
    e2e_ms, e2e_parts = p0.elapsed_time(p1), pipe_parts
    ser_value = ser_parts / (ser_ms * 1e-3)
    e2e_value = e2e_parts / (e2e_ms * 1e-3)
    if dist:
        t = torch.tensor([e2e_ms, float(e2e_parts)], dtype=torch.float64, device=dev)
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        e2e_value = t[1].item() / (tmax[0].item() * 1e-3)
    ctx2.close()

    mean_stage = {k: (sum(v) / len(v) if v else 0.0) for k, v in stage_ms.items()}
    dom = max(mean_stage, key=mean_stage.get)
    sch = ctx.get_schedule()
    roofline = (roofline_for(dom, mean_stage[dom], stats, n, desc["order"], sch["lp_fp64_pivots"], peaks,
                             sch["lp_block"], rows=bool(getattr(args, "learned", False)))
                if mean_stage[dom] > 0 else None)
    learned = None
    if args.workload == "mixture_1m" and not args.no_learned and world == 1:
        learned = learned_vs_lp(args, ctx, xb, yb, n, gi, go, h, nu, dt, total_ms / args.steps, parts / args.steps,
                                flush, stream)
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline(args.workload)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f64 (application fp32)", "data": "synthetic",
        "config": dict(desc, n_out=int(stats["n_out"]), n_diffused=int(stats["n_diffused"]),
                       n_inserted=int(stats["n_inserted"]), insertion_rounds=int(stats["rounds"]),
                       l2="flushed between steps (512 MB write)", parallelism="replicas" if world > 1 else "1 GPU"),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": args.steps, "how": "a stream of steps (vrm_step_begin / vrm_step_end on two contexts with "
                "their own buffers): every step copies its inputs in from pinned host memory and its result "
                "(gamma_out, appended positions) out on a second stream, overlapping the neighbouring steps; step "
                "k + 1 is queued before step k is waited for; one pair of events around all steps; a 512 MB L2 "
                "flush before every step, inside the timed region",
                "serial_value": ser_value, "serial_how": "each step alone (copy in, step, copy out) with an L2 "
                "flush between steps outside the events, %d steps" % e2e_steps},
        "gpu_launches": int(launches),
        "clocks": ck,
        "roofline": roofline,
        "stage_ms": {k: round(v, 4) for k, v in mean_stage.items()},
        "schedule": schedule,
        "lp": {"small_solved": int(stats["lp_small_solved"]), "small_pivots": int(stats["lp_small_pivots"]),
               "full_solved": int(stats["lp_full_solved"]), "full_pivots": int(stats["lp_full_pivots"]),
               "full_columns": int(stats["lp_full_columns"]), "max_pivots": int(stats["max_pivots"]),
               "small_ok": int(stats["small_ok"]), "full_ok": int(stats["full_ok"]),
               "no_stencil": int(stats["no_stencil"]), "small_rechecked": int(stats["lp_small_rechecked"])},
        "cpu_baseline": cpu,
        "peaks_measured": {k: round(v, 4) for k, v in peaks.items()},
    }
    if learned is not None:
        line["learned_vs_lp"] = learned
    print(json.dumps(line))
    sys.stdout.flush()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def max_moment_residual(x, y, w, n, order=1):
    """Largest max_r |sum_j V_r(xi_ij) f~_ij - b_r| over the stencils of one
    weights call (small, full and learned), in FP64 from the positions, and
    the smallest off-diagonal weight."""
    import numpy as np
    W = w["cols"].numel() // max(n, 1)
    st = w["status"][:n].cpu().numpy()
    cols = w["cols"][: n * W].view(n, W).cpu().numpy()
    f = w["f"][: n * W].view(n, W).cpu().numpy()
    sel = np.nonzero((st == 1) | (st == 2) | (st == 4))[0]
    xs, ys = x[:n].cpu().numpy(), y[:n].cpu().numpy()
    worst, fmin = 0.0, 0.0
    for a in range(0, len(sel), 1 << 18):
        s_ = sel[a:a + (1 << 18)]
        c = cols[s_]
        ok = c >= 0
        j = np.where(ok, c, 0)
        h = w["h"]
        xi = (xs[j] - xs[s_, None]) / h
        eta = (ys[j] - ys[s_, None]) / h
        ww = np.where(ok, f[s_], 0.0)
        rows = [(xi, 0.0), (eta, 0.0), (xi * xi, 2.0), (xi * eta, 0.0), (eta * eta, 2.0)]
        for r, b in rows:
            worst = max(worst, float(np.max(np.abs((r * ww).sum(1) - b))))
        fmin = min(fmin, float(np.min(ww)))
    return worst, fmin, int(len(sel))


def learned_vs_lp(args, ctx_lp, xb, yb, n, gi, go, h, nu, dt, lp_ms, lp_parts, flush, stream):
    """The second half of the metric on the same cloud and run: a network
    trained here on LP solutions (seeded jittered clouds, the learned_4m
    recipe), the step with learned stencils against the step with the LP
    alone (particles/s), acceptance, the largest moment residual and the
    smallest weight of every stencil of both, and the weak error of both on
    the heat-equation Lamb-Oseen run against the closed form."""
    import torch

    import paper_1508_06379_gb300 as vrm
    from paper_1508_06379_gb300 import learn
    t0 = time.time()
    X, T, N = learn.make_dataset(args.train_rows)
    t_data = time.time() - t0
    t0 = time.time()
    net, losses = learn.train(X, T, N, epochs=args.train_epochs, batch=4096, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    del X, T
    ctx = vrm.VRM(h=h, nu=nu)
    ctx.set_mlp(net)
    ctx.set_timing(True)
    go2 = torch.zeros_like(go)
    for _ in range(args.warmup):
        flush.zero_()
        ctx.step(xb, yb, n, gi, go2, dt)
    ms, parts, stage = 0.0, 0, {}
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n2, st = ctx.step(xb, yb, n, gi, go2, dt)
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        parts += n2
        for k, v in ctx.stage_times().items():
            stage.setdefault(k, []).append(v)
    learned_value = parts / (ms * 1e-3)
    lp_value = lp_parts / (lp_ms * 1e-3)
    # every stencil of both paths on this cloud: residual and sign
    cap = xb.numel()
    res = {}
    for name, c in (("lp", ctx_lp), ("learned", ctx)):
        x2 = torch.zeros(cap, dtype=torch.float64, device=xb.device)
        y2 = torch.zeros(cap, dtype=torch.float64, device=xb.device)
        x2[:n] = xb[:n]
        y2[:n] = yb[:n]
        n3, diff, _ = c.insert_reduce(x2, y2, n, gi)
        nb = c.build_neighbourhoods(x2, y2, n3)
        w = c.solve_weights(x2, y2, n3, diff, nb)
        w["h"] = h
        rmax, fmin, m = max_moment_residual(x2, y2, w, n3)
        res[name] = {"max_moment_residual": rmax, "min_weight": fmin, "stencils": m,
                     "learned": int(w["stats"]["learned_ok"]), "lp_small": int(w["stats"]["small_ok"]),
                     "lp_full": int(w["stats"]["full_ok"]), "none": int(w["stats"]["no_stencil"])}
    lo = lamb_oseen_weak_errors(vrm, net)
    return {
        "what": "the same cloud and run: stencils proposed by the trained network (FP64 support solve, accepted "
                "when every weight >= 0 and the moment residual <= 1e-12; LP otherwise) against the LP alone",
        "learned": {"value": learned_value, "unit": UNIT, "ms_per_step": ms / args.steps,
                    "stage_ms": {k: round(sum(v) / len(v), 4) for k, v in stage.items()},
                    "acceptance": st["learned_ok"] / max(1, st["n_diffused"]),
                    "supports_screened_per_particle": st["learned_screens"] / max(1, st["n_diffused"]),
                    **res["learned"]},
        "lp": {"value": lp_value, "unit": UNIT, "ms_per_step": lp_ms, **res["lp"]},
        "speedup_learned_over_lp": learned_value / lp_value,
        "lamb_oseen_weak_error": {"lp": lo["lp"]["weak_error"], "learned": lo["learned"]["weak_error"],
                                  "learned_fraction": lo["learned"]["learned_fraction"], "h": lo["h"],
                                  "steps": lo["lp"]["steps"]},
        "training": {"rows": int(N), "epochs": args.train_epochs, "data_s": round(t_data, 2),
                     "train_s": round(t_train, 2), "loss_first_last": [losses[0][1], losses[-1][1]]},
    }


def traffic_for(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current source of that kernel (else None)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        data = json.load(open(p))
        ent = data[kernel]
        src = open(os.path.join(ROOT, "paper_1508_06379_gb300", "csrc", ent["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest() != ent["source_sha256"]:
            return None
        return ent["bytes_per_launch"]
    except Exception:
        return None


def binding_for(kernel):
    """The kernel's busiest resources from its committed ncu capture (FP64
    pipe and issue slots as fractions of their peaks), if it was taken on the
    current source of that kernel (else None)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        ent = json.load(open(p))[kernel]
        src = open(os.path.join(ROOT, "paper_1508_06379_gb300", "csrc", ent["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest() != ent["source_sha256"]:
            return None
        return ent.get("binding")
    except Exception:
        return None


def roofline_for(stage, ms, stats, n, order=1, lp_fp64_pivots=1, peaks=None, lp_block=128, rows=False):
    m = 9 if order == 2 else 5
    if stage in ("lp_small", "lp_full"):
        if stage == "lp_small" and order == 1 and not lp_fp64_pivots:
            flops = lp_flops_certified(stats["lp_small_solved"], stats["lp_small_rechecked"],
                                       stats["lp_small_pivots"])
        elif stage == "lp_small":
            flops = lp_flops(stats["lp_small_solved"], stats["lp_small_pivots"], m)
        else:
            flops = lp_flops(stats["lp_full_solved"], stats["lp_full_pivots"], m, cols=stats["lp_full_columns"],
                             col_pivots=stats["lp_full_column_pivots"])
        kern = "k_lp_" + stage[3:]
        if stage == "lp_small" and order == 1 and not lp_fp64_pivots:
            kern = "k_lp_small32_ws" if lp_block in (192, 384) else "k_lp_small32"
        ach = flops / (ms * 1e-3) / 1e12
        if peaks and peaks.get("fp64_tflops"):
            peak = peaks["fp64_tflops"]
            src = ("of measured: FP64 FMA rate of k_fma_probe in this run (%.3f TFLOP/s; derived 152 SMs x 2 FMA "
                   "lanes/clk x 2 flop x 2.07 GHz = %.3f)" % (peak, FP64_PEAK_DERIVED_GFLOPS / 1000.0))
        else:
            peak = FP64_PEAK_DERIVED_GFLOPS / 1000.0
            src = "derived: 152 SMs x 2 FP64 FMA lanes/clk x 2 flop x 2.07 GHz"
        out = {"kernel": kern, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
               "frac": ach / peak, "traffic": traffic_for(kern) if order == 1 else None, "peak_source": src}
        binding = binding_for(kern) if order == 1 else None
        if binding:
            out["binding"] = binding
        return out
    hbm = None
    try:
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
        src = "of measured"
    except Exception:
        hbm, src = 6800.0, "of fallback"
    n_out = stats["n_out"]
    if stage == "search":
        # the step searches the diffused particles: cell key, rank and
        # cell-local position in (16 B), count, mask and small neighbourhood
        # out (37 B); the neighbour row (about 47 B more) only where the
        # learned path reads it
        nbytes = stats["n_diffused"] * (100.0 if rows else 53.0)
        kern = "k_search_all"
    elif stage == "apply":
        # Gamma in and out per target, (index, weight, source Gamma) per
        # stencil entry (at most 5 per diffused particle for n = 1) and the
        # diagonal
        nbytes = n_out * 16.0 + stats["n_diffused"] * 6 * 20.0
        kern = "k_apply_t"
    else:
        nbytes = n_out * 24.0
        kern = stage
    ach = nbytes / (ms * 1e-3) / 1e9
    return {"kernel": kern, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "traffic": traffic_for(kern), "peak_source": src}


def cpu_baseline(name, frac=1.0):
    """The oracle as it stands on a bounded sample (centred window) of the
    workload, all host cores."""
    import oracle
    oracle.build()
    x, y, g, h, nu, dt, desc = workload(name)
    if name.startswith("mixture_1m") and frac < 1.0:
        x, y, g = sample_window(x, y, g, frac)
    t0 = time.time()
    x2, y2, g2, st = oracle.step(x, y, g, h, nu, dt, order=desc["order"], R=desc["R"])
    t = time.time() - t0
    return {"value": len(x2) / t, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "one oracle step on %s of the workload (%d particles in, %d after insertion), %.1f s" % (
                "all" if frac >= 1.0 else "a centred window holding %.0f%%" % (100 * frac), len(x), len(x2), t)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    x, y, g, h, nu, dt, desc = workload(args.workload)
    frac = 0.06 if args.workload.startswith("mixture_1m") else 1.0
    if frac < 1.0:
        x, y, g = sample_window(x, y, g, frac)
    kw = dict(order=desc.get("order", 1), R=desc.get("R", 2.0))
    for _ in range(args.warmup):
        oracle.step(x, y, g, h, nu, dt, **kw)
    t0 = time.time()
    parts = 0
    for _ in range(args.steps):
        x2, y2, g2, st = oracle.step(x, y, g, h, nu, dt, **kw)
        parts += len(x2)
    t = time.time() - t0
    value = parts / t
    sample = "each step: one oracle step on the centred window holding %.0f%% of the workload (%d particles in)" % (
        100 * frac, len(x))
    cfg = dict(desc)
    if frac < 1.0:
        cfg["workload"] = ("centred window holding %.0f%% of the workload (%d particles) of: %s"
                           % (100 * frac, len(x), desc["workload"]))
        cfg["n"] = int(len(x))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


BATCH_DESC = ("64 independent jittered mixture clouds, log-uniform 1e4..5e5 particles, h ~ U[1e-3, 4e-3], "
              "jitter 0.3h, nu=1e-3, C_diff=1, insertion on, FP64, one vrm_step_batched call per step")


def batched_workload():
    import vrm_inputs
    clouds = vrm_inputs.batched_clouds()
    nu = 1e-3
    return clouds, nu, [(0.5 * h) ** 2 / (4 * nu) / 8 for (_, _, _, h) in clouds]


def run_batched(args):
    """The 64-cloud workload: one vrm_step_batched call per step (one graph
    with a branch per cloud) against the same clouds stepped one after the
    other through vrm_step (each cloud its own captured graph)."""
    import torch

    import paper_1508_06379_gb300 as vrm

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    vrm.build()
    clouds, nu, dts = batched_workload()
    dev = torch.device("cuda", local)
    devs = []
    for (x, y, g, h), dt in zip(clouds, dts):
        n = len(x)
        cap = int(n * 1.6) + 4096
        xb = torch.zeros(cap, dtype=torch.float64, device=dev)
        yb = torch.zeros(cap, dtype=torch.float64, device=dev)
        xb[:n] = torch.from_numpy(x).to(dev)
        yb[:n] = torch.from_numpy(y).to(dev)
        devs.append(dict(x=xb, y=yb, gamma_in=torch.from_numpy(g).to(dev),
                         gamma_out=torch.zeros(cap, dtype=torch.float64, device=dev), n=n, h=h, dt=dt))
    batch = vrm.VRMBatch(max_clouds=len(devs), nu=nu)
    singles = [vrm.VRM(h=d["h"], nu=nu) for d in devs]
    schedules = None
    if not args.no_autotune:
        from paper_1508_06379_gb300 import autotune
        chosen = autotune.Autotuner(args.schedule_cache).tune_batch(batch, devs)
        schedules = {}
        for k, s in chosen.items():
            schedules.setdefault("n~2^%d" % autotune.bucket(devs[k]["n"]), s)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def one_batched():
        res, st = batch.step(devs)
        return sum(r[0] for r in res), st

    def one_sequential():
        parts = 0
        for d, c in zip(devs, singles):
            n2, _ = c.step(d["x"], d["y"], d["n"], d["gamma_in"], d["gamma_out"], d["dt"], stats=False)
            parts += n2
        return parts, None

    def timed(fn, steps):
        ms, parts, st = 0.0, 0, None
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            p, s_ = fn()
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            parts += p
            st = s_ or st
        return ms, parts, st

    for _ in range(args.warmup):
        one_batched()
        one_sequential()
    torch.cuda.synchronize()
    gpu_id = None
    try:
        gpu_id = str(torch.cuda.get_device_properties(local).uuid)
        gpu_id = gpu_id if gpu_id.startswith("GPU-") else "GPU-" + gpu_id
    except Exception:
        gpu_id = None
    clocks = Clocks(gpu_id)
    time.sleep(0.5)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = vrm.launch_count()
    t_wall0 = time.time()
    ms, parts, stats = timed(one_batched, args.steps)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    launches = vrm.launch_count() - launches0
    ck = clocks.stop(t_wall0, t_wall1)
    seq_ms, seq_parts, _ = timed(one_sequential, args.steps)
    if dist:
        t = torch.tensor([ms, float(parts), seq_ms, float(seq_parts)], dtype=torch.float64, device=dev)
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        ms_max, parts_all, seq_max, seq_all = tmax[0].item(), t[1].item(), tmax[2].item(), t[3].item()
    else:
        ms_max, parts_all, seq_max, seq_all = ms, float(parts), seq_ms, float(seq_parts)
    value = parts_all / (ms_max * 1e-3)
    seq_value = seq_all / (seq_max * 1e-3)

    # end to end: host buffers in, dGamma and inserted positions out, per step
    hosts = [(torch.from_numpy(x).pin_memory(), torch.from_numpy(y).pin_memory(), torch.from_numpy(g).pin_memory(),
              torch.empty(d["x"].numel(), dtype=torch.float64).pin_memory(),
              torch.empty(d["x"].numel(), dtype=torch.float64).pin_memory(),
              torch.empty(d["x"].numel(), dtype=torch.float64).pin_memory()) for (x, y, g, _), d in zip(clouds, devs)]
    e2e_ms, e2e_parts, h2d, d2h = 0.0, 0, 0, 0
    for _ in range(max(1, min(args.steps, 5))):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for d, (xh, yh, gh, _, _, _) in zip(devs, hosts):
            n = d["n"]
            d["x"][:n].copy_(xh, non_blocking=True)
            d["y"][:n].copy_(yh, non_blocking=True)
            d["gamma_in"].copy_(gh, non_blocking=True)
        res, _ = batch.step(devs, stats=False)
        h2d = d2h = 0
        for d, (n2, _), (_, _, _, go_h, xo_h, yo_h) in zip(devs, res, hosts):
            n = d["n"]
            go_h[:n2].copy_(d["gamma_out"][:n2], non_blocking=True)
            xo_h[n:n2].copy_(d["x"][n:n2], non_blocking=True)
            yo_h[n:n2].copy_(d["y"][n:n2], non_blocking=True)
            h2d += 24 * n
            d2h += 8 * n2 + 16 * (n2 - n)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
        e2e_parts += sum(r[0] for r in res)
    e2e_value = e2e_parts / (e2e_ms * 1e-3)
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    ns = [d["n"] for d in devs]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": BATCH_DESC, "clouds": len(devs), "n_total": int(sum(ns)), "n_min": int(min(ns)),
                   "n_max": int(max(ns)), "nu": nu, "n_out": int(stats["n_out"]),
                   "n_diffused": int(stats["n_diffused"]), "n_inserted": int(stats["n_inserted"]),
                   "l2": "flushed between steps (512 MB write)", "parallelism": "replicas" if world > 1 else "1 GPU"},
        "sequential": {"value": seq_value, "unit": UNIT, "ms_per_step": seq_max / args.steps,
                       "what": "the same clouds through vrm_step one after the other, each its own captured graph "
                               "with the default schedule"},
        "schedules": schedules,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": ck,
        "roofline": None,
        "lp": {"small_solved": int(stats["lp_small_solved"]), "small_pivots": int(stats["lp_small_pivots"]),
               "full_solved": int(stats["lp_full_solved"]), "full_pivots": int(stats["lp_full_pivots"]),
               "full_columns": int(stats["lp_full_columns"]), "max_pivots": int(stats["max_pivots"]),
               "small_ok": int(stats["small_ok"]), "full_ok": int(stats["full_ok"]),
               "no_stencil": int(stats["no_stencil"]), "small_rechecked": int(stats["lp_small_rechecked"])},
        "cpu_baseline": None,
    }
    print(json.dumps(line))
    sys.stdout.flush()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


LEARNED_DESC = ("jittered lattice %dx%d (h=1e-3, jitter 0.3h), 8-Gaussian mixture, nu=1e-3, C_diff=1, insertion "
                "on; stencils from the trained network (corrected, LP fallback) vs the LP alone")


def lamb_oseen_weak_errors(vrm, net, h=1 / 128):
    """Heat-equation Lamb-Oseen run (Gamma = 1, nu = 1e-3, t = 1 -> 1.125, Euler
    with dt = (1/8)(r h)^2/(4 nu)) with the LP stencils and with the learned
    ones; the weak error against the closed form (Gaussian test functions of
    width 0.03 at five centres) of both."""
    import numpy as np
    import torch

    import vrm_inputs
    gamma, nu, t0, t1 = 1.0, 1e-3, 1.0, 1.125
    centres = [(0.0, 0.0), (0.03, 0.0), (0.05, 0.04), (-0.08, 0.02), (0.0, -0.1)]
    out = {}
    for name in ("lp", "learned"):
        x, y, g = vrm_inputs.lamb_oseen_lattice(h, gamma, nu, t0, eps=1e-8)
        dt = (0.5 * h) ** 2 / (4 * nu) / 8
        steps = int(round((t1 - t0) / dt))
        dt = (t1 - t0) / steps
        ctx = vrm.VRM(h=h, nu=nu)
        if name == "learned":
            ctx.set_mlp(net)
        n = len(x)
        cap = 8 * n + 4096
        xb = torch.zeros(cap, dtype=torch.float64, device="cuda")
        yb = torch.zeros(cap, dtype=torch.float64, device="cuda")
        xb[:n] = torch.from_numpy(x).cuda()
        yb[:n] = torch.from_numpy(y).cuda()
        bufs = [torch.zeros(cap, dtype=torch.float64, device="cuda") for _ in range(2)]
        bufs[0][:n] = torch.from_numpy(g).cuda()
        learned = diffused = 0
        for k in range(steps):
            n, st = ctx.step(xb, yb, n, bufs[k % 2], bufs[(k + 1) % 2], dt)
            learned += st["learned_ok"]
            diffused += st["n_diffused"]
        X, Y, G = xb[:n].cpu().numpy(), yb[:n].cpu().numpy(), bufs[steps % 2][:n].cpu().numpy()
        s2 = 2 * nu * t1 + 0.03 ** 2
        err = max(abs(np.sum(G * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * 0.03 ** 2))) -
                      gamma * 0.03 ** 2 / s2 * np.exp(-(cx * cx + cy * cy) / (2 * s2))) / gamma
                  for cx, cy in centres)
        out[name] = {"weak_error": float(err), "steps": steps, "n_final": int(n),
                     "learned_fraction": learned / max(1, diffused)}
    out["h"] = h
    return out


def run_learned(args):
    """The 4M-particle cloud stepped with the learned proposal and with the LP
    alone: throughput of both, acceptance, and how far the two results are
    apart (both are valid discretisations; the learned stencils meet the
    moment conditions to 1e-12)."""
    import numpy as np
    import torch

    import paper_1508_06379_gb300 as vrm
    import vrm_inputs
    from paper_1508_06379_gb300 import learn

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    vrm.build()
    dev = torch.device("cuda", local)
    t0 = time.time()
    X, T, N = learn.make_dataset(args.train_rows)
    t_data = time.time() - t0
    t0 = time.time()
    net, losses = learn.train(X, T, N, epochs=args.train_epochs, batch=4096, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    del X, T
    h, nu = 1e-3, 1e-3
    side = args.learned_side
    x, y, g = vrm_inputs.gaussian_mixture_cloud(h=h, side=side, jitter=0.3, seed=vrm_inputs.SEED_BASE + 4,
                                                half_width=0.5 * (side - 1) * h)
    dt = (0.5 * h) ** 2 / (4 * nu) / 8
    n = len(x)
    cap = int(n * 1.6) + 4096
    xb = torch.zeros(cap, dtype=torch.float64, device=dev)
    yb = torch.zeros(cap, dtype=torch.float64, device=dev)
    xb[:n] = torch.from_numpy(x).to(dev)
    yb[:n] = torch.from_numpy(y).to(dev)
    gi = torch.from_numpy(g).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    out = {}
    for name in ("lp", "learned"):
        ctx = vrm.VRM(h=h, nu=nu)
        if name == "learned":
            ctx.set_mlp(net)
        ctx.set_timing(True)
        go = torch.zeros(cap, dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            ctx.step(xb, yb, n, gi, go, dt)
        ms, parts, stage = 0.0, 0, {}
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            n2, st = ctx.step(xb, yb, n, gi, go, dt)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            parts += n2
            for k, v in ctx.stage_times().items():
                stage.setdefault(k, []).append(v)
        out[name] = dict(value=parts / (ms * 1e-3), ms=ms / args.steps, stats=st, n2=n2, gamma=go[:n2].clone(),
                         stage={k: round(sum(v) / len(v), 4) for k, v in stage.items()})
    a, b = out["lp"], out["learned"]
    g0 = torch.zeros(a["n2"], dtype=torch.float64, device=dev)
    g0[:n] = gi
    inc_lp = a["gamma"] - g0
    inc_le = b["gamma"] - g0
    rel = float(torch.linalg.norm(inc_le - inc_lp) / torch.linalg.norm(inc_lp))
    st = b["stats"]
    line = {
        "metric": METRIC, "value": b["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": b["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 (network bf16/fp32)", "data": "synthetic",
        "config": {"workload": LEARNED_DESC % (side, side), "n": n, "n_out": int(b["n2"]), "n_diffused": int(st["n_diffused"]),
                   "h": h, "nu": nu, "dt": dt, "l2": "flushed between steps (512 MB write)",
                   "train_rows": int(N), "train_epochs": args.train_epochs, "train_loss_first_last":
                   [losses[0][1], losses[-1][1]], "data_s": round(t_data, 2), "train_s": round(t_train, 2)},
        "plain_lp": {"value": a["value"], "unit": UNIT, "ms_per_step": a["ms"], "stage_ms": a["stage"]},
        "learned": {"accepted": int(st["learned_ok"]), "rejected": int(st["learned_rejected"]),
                    "accepted_on_first_support": int(st["learned_square"]),
                    "supports_screened_per_particle": st["learned_screens"] / max(1, st["n_diffused"]),
                    "acceptance": st["learned_ok"] / max(1, st["n_diffused"]),
                    "lp_small_solved": int(st["lp_small_solved"]), "stage_ms": b["stage"],
                    "increment_rel_diff_vs_lp": rel},
        "speedup_vs_plain": b["value"] / a["value"],
        "lamb_oseen": lamb_oseen_weak_errors(vrm, net),
    }
    print(json.dumps(line))
    sys.stdout.flush()


VISCOUS_DESC = ("Lamb-Oseen vortex (Gamma=1, nu=5e-4, t0=1) on a lattice of h=%.3g, |omega|>1e-10 kept, advected by "
                "its analytic velocity, SSP-RK3 with the diffusion operator at every stage (growth control and "
                "insertion once per step), dt=min((rh)^2/(4nu), h/(4 max|u|)), FP64")


def run_viscous(args):
    """Config 5: the viscous Lamb-Oseen run with advection, vrm_rk3_step per
    step; particles/s counted after insertion, each step = three operator
    evaluations; the weak error against the closed form after the timed steps."""
    import numpy as np
    import torch

    import paper_1508_06379_gb300 as vrm
    import vrm_inputs

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    vrm.build()
    dev = torch.device("cuda", local)
    gamma, nu, t0, h = 1.0, 5e-4, 1.0, args.viscous_h
    x, y, g = vrm_inputs.lamb_oseen_lattice(h, gamma, nu, t0, eps=1e-10, lo=-0.25, hi=0.25)
    umax = 0.64 * gamma / (2 * math.pi * 2.24 * math.sqrt(nu * t0))  # peak azimuthal speed
    dt = min((0.5 * h) ** 2 / (4 * nu), 0.25 * h / umax)
    n0 = len(x)
    # insertion adds particles every step (about half of n0 in the first one:
    # on a lattice whose coordinates are not binary-exact the axis
    # neighbours fall on either side of the segment rays)
    cap = 3 * n0 + 4096
    xb = torch.zeros(cap, dtype=torch.float64, device=dev)
    yb = torch.zeros(cap, dtype=torch.float64, device=dev)
    xb[:n0] = torch.from_numpy(x).to(dev)
    yb[:n0] = torch.from_numpy(y).to(dev)
    bufs = [torch.zeros(cap, dtype=torch.float64, device=dev) for _ in range(2)]
    bufs[0][:n0] = torch.from_numpy(g).to(dev)
    ctx = vrm.VRM(h=h, nu=nu, precision=args.precision)
    train_s = None
    if args.learned:
        from paper_1508_06379_gb300 import learn
        t_tr = time.time()
        X, T, N = learn.make_dataset(args.train_rows)
        net, _ = learn.train(X, T, N, epochs=args.train_epochs, batch=4096, lr=2e-3)
        del X, T
        torch.cuda.synchronize()
        train_s = time.time() - t_tr
        ctx.set_mlp(net)
    vel = dict(gamma=gamma, nu=nu)
    stream = torch.cuda.current_stream()
    n, t, k = n0, t0, 0
    learned_ok = diffused_sum = 0
    for _ in range(args.warmup):
        n, _ = ctx.rk3_step(xb, yb, n, bufs[k % 2], bufs[(k + 1) % 2], t, dt, vel)
        t += dt
        k += 1
    torch.cuda.synchronize()
    clocks = Clocks(None)
    time.sleep(0.3)
    t_wall0 = time.time()
    launches0 = vrm.launch_count()
    ms, parts, st = 0.0, 0, None
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n, st = ctx.rk3_step(xb, yb, n, bufs[k % 2], bufs[(k + 1) % 2], t, dt, vel)
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        parts += n
        t += dt
        k += 1
        learned_ok += st["learned_ok"]
        diffused_sum += 3 * st["n_diffused"]
    t_wall1 = time.time()
    launches = vrm.launch_count() - launches0
    ck = clocks.stop(t_wall0, t_wall1)
    X, Y, G = xb[:n].cpu().numpy(), yb[:n].cpu().numpy(), bufs[k % 2][:n].cpu().numpy()
    s2 = 2 * nu * t + 0.03 ** 2
    err = max(abs(np.sum(G * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * 0.03 ** 2))) -
                  gamma * 0.03 ** 2 / s2 * np.exp(-(cx * cx + cy * cy) / (2 * s2))) / gamma
              for cx, cy in [(0.0, 0.0), (0.03, 0.0), (0.05, 0.04), (-0.08, 0.02), (0.0, -0.1)])
    # e_u (Sec. 5): L2 error of the smoothed particle velocity (eps = 3h,
    # direct sum) against the Lamb-Oseen velocity, midpoint rule on a
    # 200 x 200 grid over A = [-1.5, 1.5]^2
    gq = -1.5 + (np.arange(200) + 0.5) * 0.015
    QX, QY = np.meshgrid(gq, gq)
    qx, qy = torch.from_numpy(QX.ravel().copy()).to(dev), torch.from_numpy(QY.ravel().copy()).to(dev)
    ev = torch.cuda.Event(enable_timing=True)
    ev2 = torch.cuda.Event(enable_timing=True)
    ev.record(stream)
    uh, vh = ctx.biot_savart(xb, yb, bufs[k % 2], n, qx, qy, qx.numel(), 3 * h)
    ev2.record(stream)
    ev2.synchronize()
    bs_ms = ev.elapsed_time(ev2)
    r2 = QX.ravel() ** 2 + QY.ravel() ** 2
    kq = gamma / (2 * math.pi * r2) * -np.expm1(-r2 / (4 * nu * t))
    ue, ve = -QY.ravel() * kq, QX.ravel() * kq
    uh, vh = uh.cpu().numpy(), vh.cpu().numpy()
    e_u = math.sqrt(np.sum((uh - ue) ** 2 + (vh - ve) ** 2) / np.sum(ue ** 2 + ve ** 2))
    line = {
        "metric": METRIC, "value": parts / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f64" if args.precision == "fp64" else "f64 (application fp32)") +
                 (", learned proposal bf16" if args.learned else ""), "data": "synthetic",
        "learned": {"on": bool(args.learned), "fraction_of_stencils": learned_ok / max(1, diffused_sum),
                    "train_s": train_s},
        "e_u": {"value": e_u, "targets": int(qx.numel()), "sources": int(n), "eps": 3 * h, "direct_sum_ms": bs_ms,
                "interactions_per_s": qx.numel() * n / (bs_ms * 1e-3)},
        "config": {"workload": VISCOUS_DESC % h, "n_initial": int(n0), "n_final": int(n), "h": h, "nu": nu,
                   "dt": dt, "t_final": t, "operator_evaluations_per_step": 3,
                   "l2": "inputs larger than L2 (no flush)", "parallelism": "1 GPU"},
        "circulation_drift": float(abs(G.sum() - g.sum())),
        "weak_error_vs_closed_form": float(err),
        "stats_last_step": {k2: int(st[k2]) for k2 in ("n_diffused", "n_inserted", "small_ok", "full_ok", "no_stencil")},
        "gpu_launches": int(launches), "clocks": ck, "roofline": None, "cpu_baseline": None,
    }
    print(json.dumps(line))
    sys.stdout.flush()


REMOVAL_DESC = ("particle removal pass (vrm_remove_close) on the jittered lattice 1001x1001, h=2e-3, jitter 0.3h, "
                "8-Gaussian mixture, plus 10%% extra particles within 0.3h of existing ones carrying a U(-1,1) "
                "fraction of their circulation: %d particles in")


def removal_workload():
    import numpy as np
    import vrm_inputs
    h = 2e-3
    x, y, g = vrm_inputs.gaussian_mixture_cloud(h=h, jitter=0.3, seed=vrm_inputs.SEED_BASE + 2)
    rng = np.random.default_rng(vrm_inputs.SEED_BASE + 6)
    m = len(x) // 10
    k = rng.choice(len(x), m, replace=False)
    x = np.concatenate([x, x[k] + rng.uniform(-0.3, 0.3, m) * h])
    y = np.concatenate([y, y[k] + rng.uniform(-0.3, 0.3, m) * h])
    g = np.concatenate([g, g[k] * rng.uniform(-1, 1, m)])
    return x, y, g, h


def run_removal(args):
    """Particle removal (outlook of Sec. 6.2) on a crowded 1.1M cloud: input
    particles per second of whole passes, and the oracle's pass on the host
    cores for context."""
    import torch

    import paper_1508_06379_gb300 as vrm

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    vrm.build()
    dev = torch.device("cuda", local)
    x, y, g, h = removal_workload()
    n = len(x)
    xd, yd, gd = (torch.from_numpy(a).to(dev) for a in (x, y, g))
    ctx = vrm.VRM(h=h, nu=1e-3)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ctx.remove_close(xd, yd, gd, n)
    torch.cuda.synchronize()
    clocks = Clocks(None)
    time.sleep(0.3)
    t_wall0 = time.time()
    launches0 = vrm.launch_count()
    ms, st, k = 0.0, None, 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, _, k, st = ctx.remove_close(xd, yd, gd, n)
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
    t_wall1 = time.time()
    launches = vrm.launch_count() - launches0
    ck = clocks.stop(t_wall0, t_wall1)
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t0 = time.time()
        xo, _, _, _, _, _, _ = oracle.remove_close(x, y, g, h)
        tc = time.time() - t0
        cpu = {"value": n / tc, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": "one oracle removal pass on the whole workload (%d in, %d kept), %.2f s" % (n, len(xo), tc)}
    line = {
        "metric": "particles/s per particle-removal pass on 1 GB300", "value": n * args.steps / (ms * 1e-3),
        "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": REMOVAL_DESC % n, "n": n, "n_kept": int(k), "candidates": int(st["remove_candidates"]),
                   "h": h, "l2": "flushed between passes (512 MB write)", "parallelism": "1 GPU"},
        "gpu_launches": int(launches), "clocks": ck, "roofline": None, "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    sys.stdout.flush()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched_64":
        run_batched(args)
    elif args.workload == "learned_4m":
        run_learned(args)
    elif args.workload == "viscous_16m":
        run_viscous(args)
    elif args.workload == "removal_1m":
        run_removal(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
