"""ctypes binding of libvrm.so (the C ABI of include/vrm.h).

Argument marshalling only: every stage runs in the CUDA library.  Tensors
must be contiguous CUDA tensors of the documented dtypes; the calls are
issued on torch's current CUDA stream.  If the library is missing this module
raises; there is no fallback.
"""
import ctypes
import os

import torch

from . import builder as _build

VRM_OK = 0
VRM_ERR_ARG = 1
VRM_ERR_CAPACITY = 2
VRM_ERR_CUDA = 3
VRM_ERR_UNSUPPORTED = 4
STENCIL_W = 8    # n = 1
STENCIL_W2 = 12  # n = 2
KCAP_MAX = 32
PREC_FP64 = 0
PREC_MIXED = 1
LP_NOT_DIFFUSED, LP_SMALL, LP_FULL, LP_NONE, LP_LEARNED = 0, 1, 2, 3, 4


class Params(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("r", ctypes.c_double), ("R", ctypes.c_double), ("nu", ctypes.c_double),
                ("c_diff", ctypes.c_double), ("order", ctypes.c_int32), ("k_cap", ctypes.c_int32),
                ("max_rounds", ctypes.c_int32), ("fallback", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int64), ("n_out", ctypes.c_int64), ("n_diffused", ctypes.c_int64),
                ("n_inserted", ctypes.c_int64), ("open_segments", ctypes.c_int64), ("small_ok", ctypes.c_int64),
                ("full_ok", ctypes.c_int64), ("no_stencil", ctypes.c_int64), ("rounds", ctypes.c_int32),
                ("max_pivots", ctypes.c_int32), ("max_count", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("max_dt_ratio", ctypes.c_double), ("lp_small_solved", ctypes.c_int64),
                ("lp_small_pivots", ctypes.c_int64), ("lp_full_solved", ctypes.c_int64),
                ("lp_full_pivots", ctypes.c_int64), ("learned_ok", ctypes.c_int64),
                ("learned_rejected", ctypes.c_int64), ("learned_square", ctypes.c_int64),
                ("lp_full_columns", ctypes.c_int64), ("lp_full_column_pivots", ctypes.c_int64),
                ("learned_screens", ctypes.c_int64), ("remove_candidates", ctypes.c_int64),
                ("lp_small_rechecked", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class Cloud(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("gamma_in", ctypes.c_void_p),
                ("gamma_out", ctypes.c_void_p), ("n", ctypes.c_int32), ("capacity", ctypes.c_int32),
                ("h", ctypes.c_double), ("dt", ctypes.c_double), ("n_out", ctypes.c_int32),
                ("status", ctypes.c_int32)]


class Schedule(ctypes.Structure):
    _fields_ = [("row_cap", ctypes.c_int32), ("search_block", ctypes.c_int32), ("lp_block", ctypes.c_int32),
                ("lp_blocks_per_sm", ctypes.c_int32), ("apply_block", ctypes.c_int32),
                ("lp_fp64_pivots", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]

    FIELDS = ("row_cap", "search_block", "lp_block", "lp_blocks_per_sm", "apply_block", "lp_fp64_pivots")

    def as_dict(self):
        return {k: int(getattr(self, k)) for k in self.FIELDS}

    @classmethod
    def from_dict(cls, d):
        s = cls()
        for k in cls.FIELDS:
            setattr(s, k, int(d.get(k, 0)))
        return s


class Velocity(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("gamma", ctypes.c_double),
                ("nu", ctypes.c_double), ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("eps", ctypes.c_double)]


VEL_NONE, VEL_LAMB_OSEEN, VEL_BIOT_SAVART = 0, 1, 2


class AdamW(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("weight_decay", ctypes.c_float), ("reserved", ctypes.c_int32 * 3)]


class VRMError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, _lib_handle().vrm_status_string(status).decode(), status))


# Exported symbols and their signatures (mirrors include/vrm.h).
P = ctypes.c_void_p
I32 = ctypes.c_int32
SIGNATURES = {
    "vrm_default_params": (None, [P]),
    "vrm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "vrm_stencil_width": (ctypes.c_int32, [I32]),
    "vrm_create": (ctypes.c_int, [P, P]),
    "vrm_destroy": (None, [P]),
    "vrm_insert_reduce": (ctypes.c_int, [P, P, P, I32, I32, P, P, P, P, P]),
    "vrm_build_neighbourhoods": (ctypes.c_int, [P, P, P, I32, P, P, P, P, P, P]),
    "vrm_solve_weights": (ctypes.c_int, [P, P, P, I32, P, P, P, P, P, P, P, P, P, P]),
    "vrm_apply": (ctypes.c_int, [P, I32, I32, P, P, P, P, P, P, P, P, P]),
    "vrm_step": (ctypes.c_int, [P, P, P, I32, I32, P, P, ctypes.c_double, P, P, P]),
    "vrm_step_begin": (ctypes.c_int, [P, P, P, I32, I32, P, P, ctypes.c_double, P]),
    "vrm_step_end": (ctypes.c_int, [P, P, P]),
    "vrm_set_timing": (ctypes.c_int, [P, I32]),
    "vrm_stage_times": (ctypes.c_int, [P, P]),
    "vrm_launch_count": (ctypes.c_int64, []),
    "vrm_fma_probe": (ctypes.c_int, [I32, I32, I32, P, P, P]),
    "vrm_build_neighbourhoods_noalloc": (ctypes.c_int, [P, P, P, I32, P, P, P, P, P, P]),
    "vrm_batch_create": (ctypes.c_int, [P, I32, P]),
    "vrm_batch_destroy": (None, [P]),
    "vrm_step_batched": (ctypes.c_int, [P, P, I32, P, P]),
    "vrm_get_schedule": (ctypes.c_int, [P, P]),
    "vrm_set_schedule": (ctypes.c_int, [P, P]),
    "vrm_batch_set_schedule": (ctypes.c_int, [P, I32, P]),
    "vrm_mlp_create": (ctypes.c_int, [I32, P]),
    "vrm_mlp_destroy": (None, [P]),
    "vrm_mlp_set_params": (ctypes.c_int, [P, P, P]),
    "vrm_mlp_get_params": (ctypes.c_int, [P, P, P]),
    "vrm_mlp_forward": (ctypes.c_int, [P, P, I32, P, P]),
    "vrm_mlp_grads": (ctypes.c_int, [P, P, P, I32, P, P, P]),
    "vrm_mlp_train_step": (ctypes.c_int, [P, P, P, P, I32, P, I32, P, P]),
    "vrm_mlp_adamw": (ctypes.c_int, [P, P, P, I32, P]),
    "vrm_mlp_error": (ctypes.c_int, [P, P]),
    "vrm_set_mlp": (ctypes.c_int, [P, P]),
    "vrm_rk3_step": (ctypes.c_int, [P, P, P, I32, I32, P, P, ctypes.c_double, ctypes.c_double, P, P, P, P]),
    "vrm_biot_savart": (ctypes.c_int, [P, P, P, P, I32, P, P, I32, ctypes.c_double, P, P, P]),
    "vrm_remove_close": (ctypes.c_int, [P, P, P, P, I32, P, P, P, P, P, P]),
    "vrm_learned_features": (ctypes.c_int, [P, P, P, I32, P, I32, P, P, P, P, P]),
    "vrm_learned_project": (ctypes.c_int, [P, P, P, P, I32, P, P, P, P, P, P, P, P, P]),
    "vrm_learned_targets": (ctypes.c_int, [P, I32, P, P, P, P, P]),
}
MLP_PARAMS = 164640
MLP_IN = 128
MLP_OUT = 32
NOALLOC_MAX_N = 65536
STAGES = ("reduce", "grid", "insert", "search", "lp_small", "lp_full", "apply")

_LIB = None


def library_path():
    return _build.LIB


def _lib_handle():
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libvrm.so is not built (%s); run __graft_entry__.build() or "
                               "python -m paper_1508_06379_gb300.builder" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def launch_count():
    """Kernels the library has launched in this process."""
    return int(_lib_handle().vrm_launch_count())


def fma_peak(fp64=True, blocks=None, iters=None, reps=3):
    """Peak FMA rate of this GPU in flop/s (best of `reps` launches of
    vrm_fma_probe, timed with CUDA events on the current stream)."""
    lib = _lib_handle()
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = blocks or 8 * sms
    iters = iters or (200 if fp64 else 12800)
    sink = torch.empty(blocks + 1, dtype=torch.float64 if fp64 else torch.float32, device="cuda")
    fl = ctypes.c_double()
    best = 0.0
    for _ in range(reps + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        st = lib.vrm_fma_probe(int(bool(fp64)), int(blocks), int(iters), ctypes.c_void_p(sink.data_ptr()),
                               ctypes.byref(fl), _stream())
        e1.record()
        if st != VRM_OK:
            raise VRMError(st, "vrm_fma_probe")
        e1.synchronize()
        best = max(best, fl.value / (e0.elapsed_time(e1) * 1e-3))
    return best


def build_neighbourhoods_noalloc(x, y, n, h, r=0.5, R=2.0, k_cap=32, out=None, max_count=True):
    """vrm_build_neighbourhoods_noalloc: neighbourhoods without a context and
    without any allocation inside the library (scratch in a fixed device
    array; n <= NOALLOC_MAX_N).  Output tensors may be passed in `out`."""
    lib = _lib_handle()
    p = Params()
    lib.vrm_default_params(ctypes.byref(p))
    p.h, p.r, p.R, p.k_cap = float(h), float(r), float(R), int(k_cap)
    dev = x.device
    o = out or {}
    cnt = o.get("count", torch.empty(max(n, 1), dtype=torch.int32, device=dev))
    idx = o.get("idx", torch.empty(max(n, 1) * k_cap, dtype=torch.int32, device=dev))
    mask = o.get("mask", torch.empty(max(n, 1), dtype=torch.uint8, device=dev))
    small = o.get("small", torch.empty(max(n, 1) * 8, dtype=torch.int32, device=dev))
    mc = ctypes.c_int32(0)
    st = lib.vrm_build_neighbourhoods_noalloc(
        ctypes.byref(p), _ptr(x, torch.float64, "x", n), _ptr(y, torch.float64, "y", n), int(n),
        _ptr(cnt, torch.int32, "nbr_count", n), _ptr(idx, torch.int32, "nbr_idx", n * k_cap),
        _ptr(mask, torch.uint8, "seg_mask", n), _ptr(small, torch.int32, "small", 8 * n),
        ctypes.byref(mc) if max_count else None, _stream())
    if st != VRM_OK:
        raise VRMError(st, "vrm_build_neighbourhoods_noalloc")
    return dict(count=cnt, idx=idx, mask=mask, small=small, max_count=mc.value if max_count else None)


def load_library(build_if_missing=False):
    if build_if_missing:
        _build.build()
    return _lib_handle()


def _ptr(t, dtype, what, min_numel=0):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % what)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (what, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if t.numel() < min_numel:
        raise ValueError("%s holds %d elements, needs %d" % (what, t.numel(), min_numel))
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class VRM:
    """One context of the VRM library (parameters + scratch)."""

    def __init__(self, h, nu, r=0.5, R=2.0, c_diff=1.0, order=1, k_cap=32, max_rounds=8, fallback=True,
                 precision="fp64"):
        self.lib = _lib_handle()
        p = Params()
        self.lib.vrm_default_params(ctypes.byref(p))
        p.h, p.nu, p.r, p.R, p.c_diff = float(h), float(nu), float(r), float(R), float(c_diff)
        p.order, p.k_cap, p.max_rounds, p.fallback = int(order), int(k_cap), int(max_rounds), int(bool(fallback))
        p.precision = {"fp64": PREC_FP64, "mixed": PREC_MIXED}[precision]
        self.params = p
        self.k_cap = int(k_cap)
        self.order = int(order)
        self.W = int(self.lib.vrm_stencil_width(int(order)))  # stencil row length
        h_ = ctypes.c_void_p()
        st = self.lib.vrm_create(ctypes.byref(p), ctypes.byref(h_))
        if st != VRM_OK:
            raise VRMError(st, "vrm_create")
        self.ctx = h_

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.vrm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != VRM_OK:
            raise VRMError(st, what)

    # -- stages -------------------------------------------------------------------
    def insert_reduce(self, x, y, n, gamma, diffused=None, stats=True):
        cap = x.numel()
        if diffused is None:
            diffused = torch.empty(cap, dtype=torch.uint8, device=x.device)
        n_out = ctypes.c_int32(0)
        s = Stats()
        st = self.lib.vrm_insert_reduce(self.ctx, _ptr(x, torch.float64, "x", n), _ptr(y, torch.float64, "y", cap),
                                        int(n), int(cap), _ptr(gamma, torch.float64, "gamma", n),
                                        _ptr(diffused, torch.uint8, "diffused", cap), ctypes.byref(n_out),
                                        ctypes.byref(s) if stats else None, _stream())
        self._check(st, "vrm_insert_reduce")
        return n_out.value, diffused, s.as_dict()

    def build_neighbourhoods(self, x, y, n, out=None, max_count=True):
        dev = x.device
        o = out or {}
        cnt = o.get("count", torch.empty(n, dtype=torch.int32, device=dev))
        idx = o.get("idx", torch.empty(max(n, 1) * self.k_cap, dtype=torch.int32, device=dev))
        mask = o.get("mask", torch.empty(n, dtype=torch.uint8, device=dev))
        small = o.get("small", torch.empty(max(n, 1) * 8, dtype=torch.int32, device=dev))
        mc = ctypes.c_int32(0)
        st = self.lib.vrm_build_neighbourhoods(
            self.ctx, _ptr(x, torch.float64, "x", n), _ptr(y, torch.float64, "y", n), int(n),
            _ptr(cnt, torch.int32, "nbr_count", n), _ptr(idx, torch.int32, "nbr_idx", n * self.k_cap),
            _ptr(mask, torch.uint8, "seg_mask", n), _ptr(small, torch.int32, "small", 8 * n),
            ctypes.byref(mc) if max_count else None, _stream())
        self._check(st, "vrm_build_neighbourhoods")
        return dict(count=cnt, idx=idx, mask=mask, small=small, max_count=mc.value if max_count else None)

    def solve_weights(self, x, y, n, diffused, nb, out=None, stats=True):
        dev = x.device
        o = out or {}
        W = self.W
        cols = o.get("cols", torch.empty(max(n, 1) * W, dtype=torch.int32, device=dev))
        f = o.get("f", torch.empty(max(n, 1) * W, dtype=torch.float64, device=dev))
        fii = o.get("fii", torch.empty(max(n, 1), dtype=torch.float64, device=dev))
        status = o.get("status", torch.empty(max(n, 1), dtype=torch.uint8, device=dev))
        s = Stats()
        st = self.lib.vrm_solve_weights(
            self.ctx, _ptr(x, torch.float64, "x", n), _ptr(y, torch.float64, "y", n), int(n),
            _ptr(diffused, torch.uint8, "diffused", n), _ptr(nb["count"], torch.int32, "nbr_count", n),
            _ptr(nb["idx"], torch.int32, "nbr_idx", n * self.k_cap), _ptr(nb["small"], torch.int32, "small", 8 * n),
            _ptr(cols, torch.int32, "cols", n * W), _ptr(f, torch.float64, "f", n * W),
            _ptr(fii, torch.float64, "fii", n), _ptr(status, torch.uint8, "status", n),
            ctypes.byref(s) if stats else None, _stream())
        self._check(st, "vrm_solve_weights")
        return dict(cols=cols, f=f, fii=fii, status=status, stats=s.as_dict())

    def apply(self, n, n_gamma, gamma, diffused, nb, w, dgamma=None):
        if dgamma is None:
            dgamma = torch.empty(max(n, 1), dtype=torch.float64, device=gamma.device)
        W = self.W
        st = self.lib.vrm_apply(
            self.ctx, int(n), int(n_gamma), _ptr(gamma, torch.float64, "gamma", n_gamma),
            _ptr(diffused, torch.uint8, "diffused", n), _ptr(nb["count"], torch.int32, "nbr_count", n),
            _ptr(nb["idx"], torch.int32, "nbr_idx", n * self.k_cap), _ptr(w["cols"], torch.int32, "cols", n * W),
            _ptr(w["f"], torch.float64, "f", n * W), _ptr(w["fii"], torch.float64, "fii", n),
            _ptr(dgamma, torch.float64, "dgamma", n), _stream())
        self._check(st, "vrm_apply")
        return dgamma

    def rk3_step(self, x, y, n, gamma_in, gamma_out, t, dt, lamb_oseen=None, stats=True):
        """One SSP-RK3 step (vrm_rk3_step); lamb_oseen: dict(gamma, nu[, x0, y0])
        of the advecting Lamb-Oseen field, dict(eps=...) for the particles'
        own smoothed velocity, or None (positions stay)."""
        cap = x.numel()
        v = Velocity()
        if lamb_oseen is not None and "eps" in lamb_oseen:
            v.kind = VEL_BIOT_SAVART
            v.eps = float(lamb_oseen["eps"])
        elif lamb_oseen is not None:
            v.kind = VEL_LAMB_OSEEN
            v.gamma, v.nu = float(lamb_oseen["gamma"]), float(lamb_oseen["nu"])
            v.x0, v.y0 = float(lamb_oseen.get("x0", 0.0)), float(lamb_oseen.get("y0", 0.0))
        n_out = ctypes.c_int32(0)
        s = Stats()
        st = self.lib.vrm_rk3_step(self.ctx, _ptr(x, torch.float64, "x", n), _ptr(y, torch.float64, "y", cap),
                                   int(n), int(cap), _ptr(gamma_in, torch.float64, "gamma_in", n),
                                   _ptr(gamma_out, torch.float64, "gamma_out", cap), float(t), float(dt),
                                   ctypes.byref(v), ctypes.byref(n_out), ctypes.byref(s) if stats else None,
                                   _stream())
        self._check(st, "vrm_rk3_step")
        return n_out.value, s.as_dict()

    def remove_close(self, x, y, gamma, n):
        """Particle removal (vrm_remove_close): returns (x', y', gamma', n',
        stats) with the kept particles in index order."""
        dev = x.device
        xo = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
        yo = torch.empty_like(xo)
        go = torch.empty_like(xo)
        n_out = ctypes.c_int32(0)
        s = Stats()
        self._check(self.lib.vrm_remove_close(
            self.ctx, _ptr(x, torch.float64, "x", n), _ptr(y, torch.float64, "y", n),
            _ptr(gamma, torch.float64, "gamma", n), int(n), _ptr(xo, torch.float64, "x_out", n),
            _ptr(yo, torch.float64, "y_out", n), _ptr(go, torch.float64, "gamma_out", n), ctypes.byref(n_out),
            ctypes.byref(s), _stream()), "vrm_remove_close")
        k = n_out.value
        return xo[:k], yo[:k], go[:k], k, s.as_dict()

    def biot_savart(self, xs, ys, gamma, n, xt, yt, m, eps, u=None, v=None):
        """Smoothed Biot-Savart velocity at m targets from n sources (vrm_biot_savart)."""
        dev = xs.device
        u = u if u is not None else torch.empty(max(m, 1), dtype=torch.float64, device=dev)
        v = v if v is not None else torch.empty(max(m, 1), dtype=torch.float64, device=dev)
        self._check(self.lib.vrm_biot_savart(
            self.ctx, _ptr(xs, torch.float64, "xs", n), _ptr(ys, torch.float64, "ys", n),
            _ptr(gamma, torch.float64, "gamma", n), int(n), _ptr(xt, torch.float64, "xt", m),
            _ptr(yt, torch.float64, "yt", m), int(m), float(eps), _ptr(u, torch.float64, "u", m),
            _ptr(v, torch.float64, "v", m), _stream()), "vrm_biot_savart")
        return u[:m], v[:m]

    def set_timing(self, enable=True):
        self._check(self.lib.vrm_set_timing(self.ctx, int(bool(enable))), "vrm_set_timing")

    def set_mlp(self, net):
        """Use the network's proposals first (None: the LP for every particle)."""
        self._check(self.lib.vrm_set_mlp(self.ctx, net.net if net is not None else None), "vrm_set_mlp")
        self._mlp = net  # keep it alive while the context uses it

    def learned_features(self, x, y, list_, nb, m=None):
        """Input rows (bf16 [m rounded up to 128, 128]) and slot map (int32 [m, 32])."""
        m = int(list_.numel()) if m is None else int(m)
        dev = x.device
        X = torch.zeros(max((m + 127) // 128 * 128, 128), MLP_IN, dtype=torch.bfloat16, device=dev)
        slots = torch.empty(max(m, 1), 32, dtype=torch.int32, device=dev)
        n = x.numel()
        self._check(self.lib.vrm_learned_features(
            self.ctx, _ptr(x, torch.float64, "x", n), _ptr(y, torch.float64, "y", n), int(n),
            _ptr(list_, torch.int32, "list", m) if list_ is not None else None, m,
            _ptr(nb["count"], torch.int32, "nbr_count"), _ptr(nb["idx"], torch.int32, "nbr_idx"),
            _ptr(X, torch.bfloat16, "X"), _ptr(slots, torch.int32, "slots"), _stream()), "vrm_learned_features")
        return X, slots[:m]

    def learned_project(self, x, y, list_, slots, f0, n, small):
        """Correction and acceptance of proposals f0 (fp32 [m, 32]); stencils of
        the n-particle cloud as from solve_weights, plus the accepted count."""
        m = int(slots.shape[0])
        dev = x.device
        W = STENCIL_W
        cols = torch.full((max(n, 1) * W,), -1, dtype=torch.int32, device=dev)
        f = torch.zeros(max(n, 1) * W, dtype=torch.float64, device=dev)
        fii = torch.zeros(max(n, 1), dtype=torch.float64, device=dev)
        status = torch.zeros(max(n, 1), dtype=torch.uint8, device=dev)
        acc = ctypes.c_int32(0)
        self._check(self.lib.vrm_learned_project(
            self.ctx, _ptr(x, torch.float64, "x"), _ptr(y, torch.float64, "y"),
            _ptr(list_, torch.int32, "list", m) if list_ is not None else None, m,
            _ptr(slots.contiguous(), torch.int32, "slots", 32 * m), _ptr(f0.contiguous(), torch.float32, "f0", 32 * m),
            _ptr(small, torch.int32, "small", 8 * n), _ptr(cols, torch.int32, "cols"), _ptr(f, torch.float64, "f"), _ptr(fii, torch.float64, "fii"),
            _ptr(status, torch.uint8, "status"), ctypes.byref(acc), _stream()), "vrm_learned_project")
        return dict(cols=cols, f=f, fii=fii, status=status), acc.value

    def get_schedule(self):
        s = Schedule()
        self._check(self.lib.vrm_get_schedule(self.ctx, ctypes.byref(s)), "vrm_get_schedule")
        return s.as_dict()

    def set_schedule(self, sched):
        s = Schedule.from_dict(sched)
        self._check(self.lib.vrm_set_schedule(self.ctx, ctypes.byref(s)), "vrm_set_schedule")

    def stage_times(self):
        """Stage durations (ms) of the last step made with timing on."""
        buf = (ctypes.c_float * len(STAGES))()
        self._check(self.lib.vrm_stage_times(self.ctx, buf), "vrm_stage_times")
        return dict(zip(STAGES, list(buf)))

    def step(self, x, y, n, gamma_in, gamma_out, dt, stats=True):
        """One Euler step; x, y, gamma_out hold `capacity` = x.numel() entries."""
        cap = x.numel()
        n_out = ctypes.c_int32(0)
        s = Stats()
        st = self.lib.vrm_step(self.ctx, _ptr(x, torch.float64, "x", n), _ptr(y, torch.float64, "y", cap), int(n),
                               int(cap), _ptr(gamma_in, torch.float64, "gamma_in", n),
                               _ptr(gamma_out, torch.float64, "gamma_out", cap), float(dt), ctypes.byref(n_out),
                               ctypes.byref(s) if stats else None, _stream())
        self._check(st, "vrm_step")
        return n_out.value, s.as_dict()

    def step_begin(self, x, y, n, gamma_in, gamma_out, dt):
        """vrm_step_begin: enqueues the step and returns (step_end waits)."""
        cap = x.numel()
        st = self.lib.vrm_step_begin(self.ctx, _ptr(x, torch.float64, "x", n), _ptr(y, torch.float64, "y", cap),
                                     int(n), int(cap), _ptr(gamma_in, torch.float64, "gamma_in", n),
                                     _ptr(gamma_out, torch.float64, "gamma_out", cap), float(dt), _stream())
        self._check(st, "vrm_step_begin")

    def step_end(self, stats=True):
        """vrm_step_end: waits for the pending step; returns (n_out, stats)."""
        n_out = ctypes.c_int32(0)
        s = Stats()
        st = self.lib.vrm_step_end(self.ctx, ctypes.byref(n_out), ctypes.byref(s) if stats else None)
        self._check(st, "vrm_step_end")
        return n_out.value, s.as_dict()


class VRMBatch:
    """Many independent clouds advanced by one call (vrm_step_batched); every
    parameter but the spacing h is shared."""

    def __init__(self, max_clouds, nu, r=0.5, R=2.0, c_diff=1.0, order=1, k_cap=32, max_rounds=8, fallback=True):
        self.lib = _lib_handle()
        p = Params()
        self.lib.vrm_default_params(ctypes.byref(p))
        p.h, p.nu, p.r, p.R, p.c_diff = 1.0, float(nu), float(r), float(R), float(c_diff)
        p.order, p.k_cap, p.max_rounds, p.fallback = int(order), int(k_cap), int(max_rounds), int(bool(fallback))
        self.params = p
        self.max_clouds = int(max_clouds)
        h_ = ctypes.c_void_p()
        st = self.lib.vrm_batch_create(ctypes.byref(p), self.max_clouds, ctypes.byref(h_))
        if st != VRM_OK:
            raise VRMError(st, "vrm_batch_create")
        self.b = h_

    def close(self):
        if getattr(self, "b", None):
            self.lib.vrm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_schedule(self, slot, sched):
        s = Schedule.from_dict(sched)
        st = self.lib.vrm_batch_set_schedule(self.b, int(slot), ctypes.byref(s))
        if st != VRM_OK:
            raise VRMError(st, "vrm_batch_set_schedule")

    def step(self, clouds, stats=True, raise_on_error=True):
        """clouds: sequence of dicts with x, y, gamma_in, gamma_out (CUDA float64
        tensors, capacity = x.numel()), n, h, dt.  Returns (per-cloud list of
        (n_out, status), summed stats)."""
        arr = (Cloud * max(len(clouds), 1))()
        for k, c in enumerate(clouds):
            cap = c["x"].numel()
            n = int(c["n"])
            arr[k].x = _ptr(c["x"], torch.float64, "x", n)
            arr[k].y = _ptr(c["y"], torch.float64, "y", cap)
            arr[k].gamma_in = _ptr(c["gamma_in"], torch.float64, "gamma_in", n)
            arr[k].gamma_out = _ptr(c["gamma_out"], torch.float64, "gamma_out", cap)
            arr[k].n, arr[k].capacity = n, cap
            arr[k].h, arr[k].dt = float(c["h"]), float(c["dt"])
        s = Stats()
        st = self.lib.vrm_step_batched(self.b, arr, len(clouds), ctypes.byref(s) if stats else None, _stream())
        out = [(arr[k].n_out, arr[k].status) for k in range(len(clouds))]
        if st != VRM_OK and raise_on_error:
            raise VRMError(st, "vrm_step_batched")
        return out, s.as_dict()


def _pad_rows(n, m=128):
    return (int(n) + m - 1) // m * m


class MLP:
    """The weight-proposal network (vrm_mlp_*): tensor-core forward,
    backward and AdamW.  Parameters: one float32 vector of MLP_PARAMS."""

    def __init__(self, batch_rows=4096):
        self.lib = _lib_handle()
        h_ = ctypes.c_void_p()
        st = self.lib.vrm_mlp_create(int(batch_rows), ctypes.byref(h_))
        if st != VRM_OK:
            raise VRMError(st, "vrm_mlp_create")
        self.net = h_
        self.batch_rows = int(batch_rows)

    def close(self):
        if getattr(self, "net", None):
            self.lib.vrm_mlp_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != VRM_OK:
            raise VRMError(st, what)

    def set_params(self, theta):
        t = theta if isinstance(theta, torch.Tensor) else torch.from_numpy(theta)
        t = t.to(device="cuda", dtype=torch.float32).contiguous()
        self._check(self.lib.vrm_mlp_set_params(self.net, _ptr(t, torch.float32, "theta", MLP_PARAMS), _stream()),
                    "vrm_mlp_set_params")

    def get_params(self):
        t = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
        self._check(self.lib.vrm_mlp_get_params(self.net, _ptr(t, torch.float32, "theta", MLP_PARAMS), _stream()),
                    "vrm_mlp_get_params")
        return t

    def forward(self, X, rows=None):
        """X: CUDA bfloat16 [>= rows rounded up to 128, 128]; returns fp32 [rows, 32]."""
        rows = X.shape[0] if rows is None else int(rows)
        if X.shape[0] < _pad_rows(rows):
            Xp = torch.zeros(_pad_rows(rows), MLP_IN, dtype=torch.bfloat16, device=X.device)
            Xp[:rows] = X[:rows]
            X = Xp
        Y = torch.empty(max(rows, 1), MLP_OUT, dtype=torch.float32, device=X.device)
        self._check(self.lib.vrm_mlp_forward(self.net, _ptr(X, torch.bfloat16, "X", rows * MLP_IN), rows,
                                             _ptr(Y, torch.float32, "Y", rows * MLP_OUT), _stream()),
                    "vrm_mlp_forward")
        return Y[:rows]

    def grads(self, X, T):
        rows = X.shape[0]
        g = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
        loss = torch.empty(2, dtype=torch.float32, device="cuda")
        self._check(self.lib.vrm_mlp_grads(self.net, _ptr(X, torch.bfloat16, "X", rows * MLP_IN),
                                           _ptr(T, torch.float32, "T", rows * MLP_OUT), rows,
                                           _ptr(g, torch.float32, "grad", MLP_PARAMS),
                                           _ptr(loss, torch.float32, "loss", 2), _stream()), "vrm_mlp_grads")
        return g, float(loss[0])

    @staticmethod
    def hyper(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
        return AdamW(lr, beta1, beta2, eps, weight_decay)

    def adamw(self, grad, t, **hp):
        a = self.hyper(**hp)
        self._check(self.lib.vrm_mlp_adamw(self.net, _ptr(grad, torch.float32, "grad", MLP_PARAMS), ctypes.byref(a),
                                           int(t), _stream()), "vrm_mlp_adamw")

    def train_step(self, X_all, T_all, idx, t, loss_out=None, **hp):
        """One step on rows idx (CUDA int32) of the data set; the loss (and
        mask sum) go to loss_out (CUDA float32 [2]) if given."""
        a = self.hyper(**hp)
        rows = idx.numel() if idx is not None else X_all.shape[0]
        self._check(self.lib.vrm_mlp_train_step(
            self.net, _ptr(X_all, torch.bfloat16, "X_all"), _ptr(T_all, torch.float32, "T_all"),
            _ptr(idx, torch.int32, "batch_idx", rows) if idx is not None else None, int(rows), ctypes.byref(a),
            int(t), _ptr(loss_out, torch.float32, "loss", 2) if loss_out is not None else None, _stream()),
            "vrm_mlp_train_step")

    def check(self):
        self._check(self.lib.vrm_mlp_error(self.net, _stream()), "vrm_mlp_error")


def learned_targets(list_, slots, cols, f):
    """Training targets fp32 [m, 32]: each listed particle's stencil weight at
    each slot's particle."""
    lib = _lib_handle()
    m = int(list_.numel())
    T = torch.empty(max(m, 1), MLP_OUT, dtype=torch.float32, device=list_.device)
    st = lib.vrm_learned_targets(_ptr(list_, torch.int32, "list", m), m, _ptr(slots, torch.int32, "slots", 32 * m),
                                 _ptr(cols, torch.int32, "cols"), _ptr(f, torch.float64, "f"),
                                 _ptr(T, torch.float32, "T"), _stream())
    if st != VRM_OK:
        raise VRMError(st, "vrm_learned_targets")
    return T[:m]

