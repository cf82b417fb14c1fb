"""Autotuner of the launch schedule of vrm_step (vrm_schedule in include/vrm.h).

The schedule fixes, for the three largest kernels of a step, the threads per
block, the grid cap of the small-neighbourhood LP and how many neighbour
entries the search keeps per row (row_cap).  No schedule changes a result;
the fastest one depends on the cloud's size (tails and occupancy on small
clouds, register pressure on large ones).

Tuning is a coordinate descent over three independent groups, each timed by
its own stage of the step (CUDA events recorded inside the step's graph):

  search:   row_cap in {16, 24, 32} (only values >= the cloud's widest row)
            x search_block in {64, 128, 256}
  lp_small: lp_block in {32, 64, 128} x lp_blocks_per_sm in {4, 8, 16, 32},
            or lp_block 192 / 384 (the warp-specialised binary32 LP,
            4 + 2 warps two blocks per SM / 8 + 4 warps one block per SM),
            then lp_fp64_pivots in {0, 1} (certified binary32 pivots with
            FP64 re-runs, or FP64 pivots throughout: lattices with many
            exact ties re-run most LPs and may prefer FP64)
  apply:    apply_block in {64, 128, 256}

Every candidate's output (positions and Gamma after the step) is checked to
be bit-identical to the default schedule's; a difference is an error.
Results are cached as JSON per device, k_cap, consistency order and size
bucket (nearest power of two of the particle count); batches take the
schedule of each cloud's bucket.
"""
import json
import math
import os
import statistics

DEFAULT = dict(row_cap=32, search_block=256, lp_block=128, lp_blocks_per_sm=16, apply_block=256, lp_fp64_pivots=0)
GROUPS = (
    ("search", [dict(row_cap=r, search_block=b) for r in (16, 24, 32) for b in (64, 128, 256)]),
    ("lp_small", [dict(lp_block=b, lp_blocks_per_sm=k) for b in (32, 64, 128) for k in (4, 8, 16, 32)] +
     [dict(lp_block=192, lp_blocks_per_sm=2), dict(lp_block=384, lp_blocks_per_sm=1)]),
    ("lp_small", [dict(lp_fp64_pivots=v) for v in (0, 1)]),
    ("apply", [dict(apply_block=b) for b in (64, 128, 256)]),
)


def bucket(n):
    """Size bucket of a cloud: the nearest power of two of n."""
    return int(round(math.log2(max(int(n), 1))))


def cache_key(device, k_cap, n, order=1):
    o = "" if int(order) == 1 else "|o%d" % int(order)
    return "%s|k%d%s|n2^%d" % (device, int(k_cap), o, bucket(n))


def default_cache_path():
    p = os.environ.get("VRM_SCHEDULE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_1508_06379_gb300", "schedules.json")


def feasible(option, k_cap, max_count):
    """row_cap options below the widest row (or above k_cap) are skipped."""
    r = option.get("row_cap")
    return r is None or (max_count <= r <= k_cap)


def descend(measure, k_cap, max_count, start=None, groups=GROUPS):
    """Coordinate descent.  measure(schedule) -> (stage_ms dict, same_output
    bool).  Returns (best schedule, report list of (group, option, ms))."""
    cur = dict(start or DEFAULT)
    cur["row_cap"] = min(cur["row_cap"], k_cap)
    report = []
    for stage, options in groups:
        best_ms, best_opt = None, None
        for opt in options:
            if not feasible(opt, k_cap, max_count):
                continue
            cand = dict(cur, **opt)
            ms, same = measure(cand)
            if not same:
                raise RuntimeError("schedule %s changed the step's output" % cand)
            t = ms[stage]
            report.append((stage, opt, t))
            if best_ms is None or t < best_ms:
                best_ms, best_opt = t, opt
        if best_opt is not None:
            cur.update(best_opt)
    return cur, report


def device_name():
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s|sm%d%d" % (p.name.replace("|", "/"), p.major, p.minor)


def tune_context(ctx, x, y, n, gamma_in, gamma_out, dt, reps=5):
    """Tunes ctx's schedule on one cloud (device buffers as for VRM.step) and
    leaves the best one set.  Returns (schedule, report)."""
    import torch
    ctx.set_schedule(dict(DEFAULT, row_cap=min(DEFAULT["row_cap"], ctx.k_cap)))
    n2, st = ctx.step(x, y, n, gamma_in, gamma_out, dt)
    ref_x, ref_g = x[:n2].clone(), gamma_out[:n2].clone()
    max_count = int(st["max_count"])
    ctx.set_timing(True)

    def measure(sched):
        ctx.set_schedule(sched)
        per_stage = {}
        same = True
        for r in range(reps + 1):
            m, _ = ctx.step(x, y, n, gamma_in, gamma_out, dt, stats=False)
            times = ctx.stage_times()
            if r == 0:  # the first run captures the graph
                same = m == n2 and torch.equal(x[:m], ref_x) and torch.equal(gamma_out[:m], ref_g)
                continue
            for k, v in times.items():
                per_stage.setdefault(k, []).append(v)
        return {k: statistics.median(v) for k, v in per_stage.items()}, same

    try:
        best, report = descend(measure, ctx.k_cap, max_count)
    finally:
        ctx.set_timing(False)
    ctx.set_schedule(best)
    return best, report


class Autotuner:
    """Schedules per (device, k_cap, order, size bucket), tuned on first use
    and kept in a JSON file."""

    def __init__(self, path=None, reps=5):
        self.path = path or default_cache_path()
        self.reps = reps
        self.table = {}
        if os.path.exists(self.path):
            try:
                self.table = json.load(open(self.path))
            except (OSError, ValueError):
                self.table = {}

    def save(self):
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.table, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def lookup(self, k_cap, n, order=1):
        return self.table.get(cache_key(device_name(), k_cap, n, order))

    def schedule_for(self, ctx, cloud):
        """Cached schedule of the cloud's bucket, tuned on this cloud if
        missing.  cloud: dict with x, y, n, gamma_in, gamma_out, dt."""
        key = cache_key(device_name(), ctx.k_cap, cloud["n"], getattr(ctx, "order", 1))
        if key not in self.table:
            best, _ = tune_context(ctx, cloud["x"], cloud["y"], cloud["n"], cloud["gamma_in"], cloud["gamma_out"],
                                   cloud["dt"], self.reps)
            self.table[key] = best
            self.save()
        return self.table[key]

    def apply(self, ctx, cloud):
        s = self.schedule_for(ctx, cloud)
        ctx.set_schedule(s)
        return s

    def tune_batch(self, batch, clouds):
        """Sets every slot of `batch` to the schedule of its cloud's bucket,
        tuning each missing bucket on its largest cloud (alone, on scratch
        copies of that cloud's buffers)."""
        import torch

        from .binding import VRM
        p = batch.params
        by_bucket = {}
        for k, c in enumerate(clouds):
            if int(c["n"]) > 0:
                by_bucket.setdefault(bucket(c["n"]), []).append(k)
        chosen = {}
        for b, slots in sorted(by_bucket.items()):
            key = cache_key(device_name(), p.k_cap, clouds[slots[0]]["n"], p.order)
            if key not in self.table:
                rep = max(slots, key=lambda k: int(clouds[k]["n"]))
                c = clouds[rep]
                ctx = VRM(h=c["h"], nu=p.nu, r=p.r, R=p.R, c_diff=p.c_diff, order=p.order, k_cap=p.k_cap,
                          max_rounds=p.max_rounds, fallback=bool(p.fallback))
                xs, ys = c["x"].clone(), c["y"].clone()
                go = torch.zeros_like(c["gamma_out"])
                self.table[key], _ = tune_context(ctx, xs, ys, int(c["n"]), c["gamma_in"], go, c["dt"], self.reps)
                ctx.close()
                self.save()
            for k in slots:
                batch.set_schedule(k, self.table[key])
                chosen[k] = self.table[key]
        return chosen
