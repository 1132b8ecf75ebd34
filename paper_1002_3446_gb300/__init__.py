"""GB300-native leading-order, leading-colour multi-gluon event generator.

Thin Python binding of the C ABI in ``include/tess.h`` (``_build/libtess.so``):
argument marshalling only.  Every step of an event runs in the library's
CUDA kernels; PyTorch is used for device memory and streams.  There is no
CPU path: if the CUDA library cannot be loaded, every call raises.

Names follow the C ABI (``tess_init``, ``tess_generate``, ...).  ``n`` is the
total number of gluons (gg -> (n-2) g), as in the paper.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libtess.so")

TESS_OK = 0
TESS_E_INVALID = -1
TESS_E_UNSUPPORTED = -2
TESS_E_CUDA = -3
TESS_E_WORKSPACE = -4
TESS_E_NUMERICAL = -5
TESS_MIN_N, TESS_MAX_N, TESS_MAX_BINS, TESS_ACC_LEN = 4, 12, 1024, 8
TESS_NOALLOC_SCRATCH_BYTES, TESS_NOALLOC_MAX_BINS = 1 << 20, 254
TESS_FP64, TESS_FP32_CURRENTS, TESS_FP32_DS = 0, 1, 2
TESS_HEL_SUM, TESS_HEL_SAMPLE, TESS_POL_RANDOM = 0, 1, 2
TESS_FLAG_CUT_FIRST, TESS_FLAG_PDF_GRID = 1, 2
TESS_OBS_PTLEAD, TESS_OBS_HT, TESS_OBS_RMIN = 0, 1, 2
TESS_K2_REG, TESS_K2_ROWS32, TESS_K2_ROWS64, TESS_K2_LOOP, TESS_K2_REG_HI, TESS_K2_REG_TMA = 0, 1, 2, 3, 4, 5
TESS_K2_REG_TMA_HI, TESS_K2_PAIR32, TESS_K2_PAIR64, TESS_K2_REAL, TESS_K2_REAL_HI = 6, 7, 8, 9, 10
TESS_K2_ROWS_REAL, TESS_K2_PAIR_W, TESS_K2_WAVE, TESS_K2_WAVE2, TESS_K2_WAVE2U = 11, 12, 13, 14, 15
TESS_K2_WAVE2P, TESS_K2_WAVE2PU, TESS_K2_WAVE2L, TESS_K2_REG_HI4, TESS_K2_REG_HI_PF = 16, 17, 18, 19, 20
TESS_K2_LANES8, TESS_K2_LANES16, TESS_K2_LANES32 = 21, 22, 23
TESS_K2_FUSED = 24
TESS_SCHED_SERIAL, TESS_SCHED_OVERLAP, TESS_SCHED_OVERLAP_TILES, TESS_SCHED_SERIAL_TILES = 0, 1, 2, 3
TESS_SCHED_SERIAL_HIST = 4
TESS_PEAK_FP32, TESS_PEAK_FP32X2, TESS_PEAK_FP64 = 0, 1, 2

# Every symbol include/tess.h declares (checked by the ABI tests).
EXPORTED = ["tess_version", "tess_last_error", "tess_init", "tess_destroy", "tess_workspace_size", "tess_generate",
            "tess_me2", "tess_result", "tess_weights", "tess_histograms", "tess_generate_noalloc",
            "tess_kernel_launches", "tess_workspace_size_batched", "tess_generate_batched", "tess_autotune",
            "tess_stage_timing", "tess_stage_times", "tess_draws", "tess_gradients", "tess_select_variant",
            "tess_plan_info", "tess_gradients_workspace_size", "tess_gauge_ratio", "tess_peak_flops",
            "tess_workspace_size_persistent", "tess_generate_persistent", "tess_autotune_outputs",
            "tess_set_chunk_bytes"]


class TessError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tess error {code}: {msg}")
        self.code = code


class tess_process(ctypes.Structure):
    _fields_ = [
        ("n_gluons", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("helicity_mode", ctypes.c_int32),
        ("hist_observable", ctypes.c_int32),
        ("hist_bins", ctypes.c_int32),
        ("nf", ctypes.c_int32),
        ("sqrt_s", ctypes.c_double),
        ("pt_min", ctypes.c_double),
        ("eta_max", ctypes.c_double),
        ("dr_min", ctypes.c_double),
        ("alphas_mz", ctypes.c_double),
        ("mz", ctypes.c_double),
        ("mu_r_factor", ctypes.c_double),
        ("hist_lo", ctypes.c_double),
        ("hist_hi", ctypes.c_double),
        ("flags", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class tess_outputs(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in ("weight", "me2", "pass_", "ht", "ptlead", "rmin", "acc", "hist")]


_lock = threading.Lock()
_lib = None


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            from . import build as _build
            _build.build()
        lib = ctypes.CDLL(_LIB_PATH)
        vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
        P = ctypes.POINTER
        lib.tess_version.restype = ctypes.c_char_p
        lib.tess_last_error.restype = ctypes.c_char_p
        lib.tess_init.argtypes = [i32, P(vp)]
        lib.tess_destroy.argtypes = [vp]
        lib.tess_destroy.restype = None
        lib.tess_workspace_size.argtypes = [vp, P(tess_process), u64, P(ctypes.c_size_t)]
        lib.tess_kernel_launches.argtypes = [vp, P(tess_process), u64, P(ctypes.c_int)]
        lib.tess_workspace_size_batched.argtypes = [vp, i32, P(tess_process), P(u64), P(ctypes.c_size_t)]
        lib.tess_generate_batched.argtypes = [vp, i32, P(tess_process), P(u64), P(u64), P(u64), P(tess_outputs), vp,
                                              ctypes.c_size_t, vp]
        lib.tess_workspace_size_persistent.argtypes = [vp, i32, P(tess_process), P(u64), P(ctypes.c_size_t)]
        lib.tess_generate_persistent.argtypes = [vp, i32, P(tess_process), P(u64), P(u64), P(u64), P(tess_outputs),
                                                 vp, ctypes.c_size_t, vp]
        lib.tess_autotune.argtypes = [vp, P(tess_process), u64, vp, vp, ctypes.c_size_t, vp, P(ctypes.c_int)]
        lib.tess_autotune_outputs.argtypes = [vp, P(tess_process), u64, P(tess_outputs), vp, ctypes.c_size_t, vp,
                                              P(ctypes.c_int)]
        lib.tess_stage_timing.argtypes = [vp, i32]
        lib.tess_select_variant.argtypes = [vp, P(tess_process), i32, i32]
        lib.tess_set_chunk_bytes.argtypes = [vp, ctypes.c_size_t]
        lib.tess_plan_info.argtypes = [vp, P(tess_process), u64, P(ctypes.c_int)]
        lib.tess_draws.argtypes = [vp, i32, u64, u64, u64, vp, vp, vp, vp]
        lib.tess_gradients.argtypes = [vp, P(tess_process), u64, vp, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_size_t,
                                       vp]
        lib.tess_gradients_workspace_size.argtypes = [vp, P(tess_process), u64, P(ctypes.c_size_t)]
        lib.tess_stage_times.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_int)]
        lib.tess_generate.argtypes = [vp, P(tess_process), u64, u64, u64, P(tess_outputs), vp, ctypes.c_size_t, vp]
        lib.tess_me2.argtypes = [vp, i32, i32, u64, vp, vp, vp, vp, vp]
        lib.tess_gauge_ratio.argtypes = [vp, i32, i32, u64, vp, vp, vp, vp, vp]
        lib.tess_generate_noalloc.argtypes = [vp, P(tess_process), u64, u64, u64, P(tess_outputs), vp]
        lib.tess_result.argtypes = [vp, vp, P(ctypes.c_double), vp]
        lib.tess_weights.argtypes = [vp, P(tess_outputs), u64, vp, vp, vp, vp]
        lib.tess_histograms.argtypes = [vp, P(tess_process), vp, vp, vp, vp]
        lib.tess_peak_flops.argtypes = [vp, i32, i32, P(ctypes.c_double), vp]
        for f in EXPORTED:
            if f not in ("tess_version", "tess_last_error", "tess_destroy"):
                getattr(lib, f).restype = i32
        _lib = lib
        return lib


def library_path():
    return _LIB_PATH


def _check(rc):
    if rc != TESS_OK:
        raise TessError(rc, _load().tess_last_error().decode())
    return rc


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ----------------------------------------------------------------- C ABI
def tess_version():
    return _load().tess_version().decode()


def tess_last_error():
    return _load().tess_last_error().decode()


def tess_init(device=0):
    h = ctypes.c_void_p()
    _check(_load().tess_init(int(device), ctypes.byref(h)))
    return h


def tess_destroy(ctx):
    _load().tess_destroy(ctx)


def tess_workspace_size(ctx, proc, n_events):
    b = ctypes.c_size_t()
    _check(_load().tess_workspace_size(ctx, ctypes.byref(proc), int(n_events), ctypes.byref(b)))
    return b.value


def tess_kernel_launches(ctx, proc, n_events):
    c = ctypes.c_int()
    _check(_load().tess_kernel_launches(ctx, ctypes.byref(proc), int(n_events), ctypes.byref(c)))
    return c.value


def _u64s(xs):
    return (ctypes.c_uint64 * len(xs))(*[int(x) for x in xs])


def tess_workspace_size_batched(ctx, procs, n_events):
    arr = (tess_process * len(procs))(*procs)
    b = ctypes.c_size_t()
    _check(_load().tess_workspace_size_batched(ctx, len(procs), arr, _u64s(n_events), ctypes.byref(b)))
    return b.value


def tess_generate_batched(ctx, procs, seeds, first_events, n_events, outputs, workspace, stream=None):
    k = len(procs)
    arr = (tess_process * k)(*procs)
    outs = (tess_outputs * k)(*outputs)
    nbytes = workspace.numel() * workspace.element_size()
    _check(_load().tess_generate_batched(ctx, k, arr, _u64s(seeds), _u64s(first_events), _u64s(n_events), outs,
                                         _ptr(workspace), nbytes, _stream(stream)))


def tess_workspace_size_persistent(ctx, procs, n_events):
    arr = (tess_process * len(procs))(*procs)
    b = ctypes.c_size_t()
    _check(_load().tess_workspace_size_persistent(ctx, len(procs), arr, _u64s(n_events), ctypes.byref(b)))
    return b.value


def tess_generate_persistent(ctx, procs, seeds, first_events, n_events, outputs, workspace, stream=None):
    k = len(procs)
    arr = (tess_process * k)(*procs)
    outs = (tess_outputs * k)(*outputs)
    nbytes = workspace.numel() * workspace.element_size()
    _check(_load().tess_generate_persistent(ctx, k, arr, _u64s(seeds), _u64s(first_events), _u64s(n_events), outs,
                                            _ptr(workspace), nbytes, _stream(stream)))


def tess_autotune(ctx, proc, probe_events, acc_scratch, workspace, stream=None, outputs=None):
    """Times every amplitude variant and schedule on probe_events events and keeps the fastest.
    With `outputs` (a tess_outputs, e.g. Run.outputs, per-event arrays of at least probe_events
    entries) the timed runs write those per-event arrays as the later calls will
    (tess_autotune_outputs); acc_scratch is then unused."""
    f = ctypes.c_int()
    nbytes = workspace.numel() * workspace.element_size()
    if outputs is not None:
        _check(_load().tess_autotune_outputs(ctx, ctypes.byref(proc), int(probe_events), ctypes.byref(outputs),
                                             _ptr(workspace), nbytes, _stream(stream), ctypes.byref(f)))
    else:
        _check(_load().tess_autotune(ctx, ctypes.byref(proc), int(probe_events), _ptr(acc_scratch),
                                     _ptr(workspace), nbytes, _stream(stream), ctypes.byref(f)))
    return f.value


def tess_select_variant(ctx, proc, form=-1, schedule=-1):
    _check(_load().tess_select_variant(ctx, ctypes.byref(proc), int(form), int(schedule)))


def tess_set_chunk_bytes(ctx, nbytes):
    """Bytes of per-event intermediate data per chunk of the sampled-event pipeline (0: default, 4 GiB)."""
    _check(_load().tess_set_chunk_bytes(ctx, int(nbytes)))


def tess_plan_info(ctx, proc, n_events):
    """Amplitude variant, schedule in effect, chunks and amplitude grid of a call with n_events."""
    info = (ctypes.c_int * 4)()
    _check(_load().tess_plan_info(ctx, ctypes.byref(proc), int(n_events), info))
    return {"variant": info[0], "schedule": info[1], "chunks": info[2], "grid": info[3]}


STAGES = ("kinematics", "amplitude", "finalize", "fused")


def tess_stage_timing(ctx, enable):
    _check(_load().tess_stage_timing(ctx, int(bool(enable))))


def tess_stage_times(ctx):
    ms = (ctypes.c_double * 4)()
    n = (ctypes.c_int * 4)()
    _check(_load().tess_stage_times(ctx, ms, n))
    return {STAGES[i]: (ms[i], n[i]) for i in range(4)}


def n_uniforms(n):
    """x1, x2 and four Rambo uniforms per final-state gluon."""
    return 2 + 4 * (n - 2)


def tess_draws(ctx, n, seed, first_event, n_events, stream=None):
    """The generator's own random inputs (u, hel, order) of an event range."""
    import torch
    u = torch.empty((n_events, n_uniforms(n)), dtype=torch.float64, device="cuda")
    hel = torch.empty(n_events, dtype=torch.int32, device="cuda")
    order = torch.empty((n_events, n), dtype=torch.uint8, device="cuda")
    _check(_load().tess_draws(ctx, int(n), int(seed), int(first_event), int(n_events), _ptr(u), _ptr(hel),
                              _ptr(order), _stream(stream)))
    return u, hel, order


def tess_gradients_workspace_size(ctx, proc, n_events):
    b = ctypes.c_size_t()
    _check(_load().tess_gradients_workspace_size(ctx, ctypes.byref(proc), int(n_events), ctypes.byref(b)))
    return b.value


def tess_gradients(ctx, proc, u, hel, order, dL_dw=None, want=("w", "dw_du", "dw_dk", "dw_dlnmu"), stream=None,
                   workspace=None):
    """Event weights and their gradients (see include/tess.h); returns a dict of
    device tensors for the requested outputs.  workspace: a device tensor of
    at least tess_gradients_workspace_size bytes (allocated here if None)."""
    import torch
    E = u.shape[0]
    n = proc.n_gluons
    f64 = dict(dtype=torch.float64, device=u.device)
    out = {"w": torch.empty(E, **f64) if "w" in want else None,
           "dw_du": torch.empty((E, n_uniforms(n)), **f64) if "dw_du" in want else None,
           "dw_dk": torch.empty((E, n, 4), **f64) if "dw_dk" in want else None,
           "dw_dlnmu": torch.empty(E, **f64) if "dw_dlnmu" in want else None}
    if workspace is None:
        need = tess_gradients_workspace_size(ctx, proc, E)
        workspace = torch.empty((need + 7) // 8, **f64) if need else None
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(_load().tess_gradients(ctx, ctypes.byref(proc), int(E), _ptr(u.contiguous()), _ptr(hel), _ptr(order),
                                  _ptr(dL_dw), _ptr(out["w"]), _ptr(out["dw_du"]), _ptr(out["dw_dk"]),
                                  _ptr(out["dw_dlnmu"]), _ptr(workspace), nbytes, _stream(stream)))
    return {k: v for k, v in out.items() if v is not None}


def _weight_function():
    import torch

    class EventWeight(torch.autograd.Function):
        """w(u, log_xi) for fixed helicity labels and colour orderings, with
        mu_R = xi H_T / 2; the backward pass is the library's adjoint kernel
        (a vector-Jacobian product with the upstream gradient)."""

        @staticmethod
        def forward(fctx, u, log_xi, tctx, proc, hel, order):
            p = tess_process.from_buffer_copy(proc)
            p.mu_r_factor = proc.mu_r_factor * float(torch.exp(log_xi))
            fctx.save_for_backward(u)
            fctx.meta = (tctx, p, hel, order)
            return tess_gradients(tctx, p, u.detach(), hel, order, want=("w",))["w"]

        @staticmethod
        def backward(fctx, grad_w):
            (u,) = fctx.saved_tensors
            tctx, p, hel, order = fctx.meta
            g = tess_gradients(tctx, p, u.detach(), hel, order, dL_dw=grad_w.contiguous(),
                               want=("dw_du", "dw_dlnmu"))
            return g["dw_du"], g["dw_dlnmu"].sum().reshape(()), None, None, None, None

    return EventWeight


def event_weight(tctx, proc, u, hel, order, log_xi=None):
    """Differentiable event weights: torch.autograd sees w as a function of the
    uniforms u (and of log_xi = ln(mu_R / (H_T/2)) when given)."""
    import torch
    if log_xi is None:
        log_xi = torch.zeros((), dtype=torch.float64, device=u.device)
    return _weight_function().apply(u, log_xi, tctx, proc, hel, order)


def make_outputs(weight=None, me2=None, pass_=None, ht=None, ptlead=None, rmin=None, acc=None, hist=None):
    return tess_outputs(*[t.data_ptr() if t is not None else None for t in (weight, me2, pass_, ht, ptlead, rmin,
                                                                            acc, hist)])


def tess_generate(ctx, proc, seed, first_event, n_events, outputs, workspace, stream=None):
    ws = _ptr(workspace)
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(_load().tess_generate(ctx, ctypes.byref(proc), int(seed), int(first_event), int(n_events),
                                 ctypes.byref(outputs), ws, nbytes, _stream(stream)))


def tess_peak_flops(ctx, kind, reps=5, stream=None):
    """Measured FMA rate (TFLOP/s) of kind TESS_PEAK_FP32 / _FP32X2 / _FP64."""
    t = ctypes.c_double()
    _check(_load().tess_peak_flops(ctx, int(kind), int(reps), ctypes.byref(t), _stream(stream)))
    return t.value


def tess_generate_noalloc(ctx, proc, seed, first_event, n_events, outputs, stream=None):
    """tess_generate without a workspace: for callers that cannot allocate
    device memory (the scratch lives in a fixed array inside the library)."""
    _check(_load().tess_generate_noalloc(ctx, ctypes.byref(proc), int(seed), int(first_event), int(n_events),
                                         ctypes.byref(outputs), _stream(stream)))


def tess_me2(ctx, n, precision, k, order, hel, me2, stream=None):
    _check(_load().tess_me2(ctx, int(n), int(precision), int(me2.numel()), _ptr(k), _ptr(order), _ptr(hel),
                            _ptr(me2), _stream(stream)))


def tess_gauge_ratio(ctx, n, precision, k, order, hel, ratio, stream=None):
    _check(_load().tess_gauge_ratio(ctx, int(n), int(precision), int(ratio.numel()), _ptr(k), _ptr(order), _ptr(hel),
                                    _ptr(ratio), _stream(stream)))


def tess_result(ctx, acc, stream=None, allow_nonfinite=False):
    out = (ctypes.c_double * 4)()
    rc = _load().tess_result(ctx, _ptr(acc), out, _stream(stream))
    if rc != TESS_OK and not (allow_nonfinite and rc == TESS_E_NUMERICAL):
        _check(rc)
    return out[0], out[1], int(out[2]), int(out[3])


def tess_weights(ctx, outputs, n_events, host_weight=None, host_pass=None, host_me2=None, stream=None):
    def hp(a):
        return None if a is None else ctypes.c_void_p(a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr())
    _check(_load().tess_weights(ctx, ctypes.byref(outputs), int(n_events), hp(host_weight), hp(host_pass),
                                hp(host_me2), _stream(stream)))


def tess_histograms(ctx, proc, hist, stream=None):
    nb2 = proc.hist_bins + 2
    sw = np.zeros(nb2)
    sw2 = np.zeros(nb2)
    _check(_load().tess_histograms(ctx, ctypes.byref(proc), _ptr(hist), ctypes.c_void_p(sw.ctypes.data),
                                   ctypes.c_void_p(sw2.ctypes.data), _stream(stream)))
    return sw, sw2


# ----------------------------------------------------------------- helpers
def process(n, precision=TESS_FP64, helicity_mode=TESS_HEL_SAMPLE, sqrt_s=14000.0, pt_min=20.0, eta_max=2.5,
            dr_min=0.4, alphas_mz=0.118, mz=91.19, nf=5, mu_r_factor=0.5, hist_observable=TESS_OBS_PTLEAD,
            hist_bins=0, hist_lo=20.0, hist_hi=1020.0, flags=0):
    return tess_process(n_gluons=n, precision=precision, helicity_mode=helicity_mode,
                        hist_observable=hist_observable, hist_bins=hist_bins, nf=nf, sqrt_s=sqrt_s, pt_min=pt_min,
                        eta_max=eta_max, dr_min=dr_min, alphas_mz=alphas_mz, mz=mz, mu_r_factor=mu_r_factor,
                        hist_lo=hist_lo, hist_hi=hist_hi, flags=flags, reserved=0)


# Workloads of the numerical study (Sec. 4), 14 TeV, toy gluon density.
PRESETS = {
    "gg2g": dict(n=4, precision=TESS_FP64, helicity_mode=TESS_HEL_SUM, hist_observable=TESS_OBS_PTLEAD,
                 hist_bins=50, hist_lo=20.0, hist_hi=1020.0, n_events=1 << 20),
    "gg4g": dict(n=6, precision=TESS_FP32_CURRENTS, helicity_mode=TESS_HEL_SAMPLE, n_events=1 << 24),
    "gg8g": dict(n=10, precision=TESS_FP32_CURRENTS, helicity_mode=TESS_HEL_SAMPLE, pt_min=30.0,
                 hist_observable=TESS_OBS_HT, hist_bins=40, hist_lo=200.0, hist_hi=3000.0, n_events=1 << 26),
}


class Run:
    """Device buffers (torch) for one call of tess_generate plus its
    accumulators; ``per_event`` selects which per-event arrays exist."""

    def __init__(self, ctx, proc, n_events, device="cuda", per_event=("weight", "me2", "pass", "ht", "ptlead", "rmin"),
                 host_per_event=False):
        """host_per_event: the per-event arrays are pinned host memory, which
        the kernels write directly (no device-to-host copy afterwards)."""
        import torch
        self.ctx, self.proc, self.n_events = ctx, proc, int(n_events)
        dev = torch.device(device)
        f64 = dict(dtype=torch.float64, device=dev)

        def per_event_array(dtype):
            if host_per_event:
                return torch.empty(self.n_events, dtype=dtype).pin_memory()
            return torch.empty(self.n_events, dtype=dtype, device=dev)

        self.t = {}
        for name in ("weight", "me2", "ht", "ptlead", "rmin"):
            self.t[name] = per_event_array(torch.float64) if name in per_event else None
        self.t["pass"] = per_event_array(torch.uint8) if "pass" in per_event else None
        self.acc = torch.zeros(TESS_ACC_LEN, **f64)
        self.hist = torch.zeros(4 * (proc.hist_bins + 2), **f64) if proc.hist_bins > 0 else None
        ws = tess_workspace_size(ctx, proc, self.n_events)
        self.workspace = torch.empty((ws + 7) // 8, **f64)
        self.outputs = make_outputs(self.t["weight"], self.t["me2"], self.t["pass"], self.t["ht"], self.t["ptlead"],
                                    self.t["rmin"], self.acc, self.hist)

    def reset(self):
        self.acc.zero_()
        if self.hist is not None:
            self.hist.zero_()

    def generate(self, seed, first_event=0, stream=None):
        tess_generate(self.ctx, self.proc, seed, first_event, self.n_events, self.outputs, self.workspace, stream)

    def result(self, stream=None, allow_nonfinite=False):
        return tess_result(self.ctx, self.acc, stream, allow_nonfinite)

    def histograms(self, stream=None):
        return tess_histograms(self.ctx, self.proc, self.hist, stream)


# ----------------------------------------------------------------- cost model
def bg_flops(n):
    """Real floating-point operations (FMA = 2, add/mul/reciprocal = 1) of one
    Berends-Giele amplitude as the kernels evaluate it (tess_bg.cuh): per
    split 148 (+2 for each S term of a multi-leg side), per four-vertex triple
    62, per set 20 plus 16 when propagated, and the final contraction 30."""
    L = n - 1
    total = 0
    for ln in range(2, L + 1):
        for a in range(0, L - ln + 1):
            b = a + ln - 1
            for i in range(a, b):
                total += 148 + (2 if i > a else 0) + (2 if b > i + 1 else 0)
            total += 62 * ((ln - 1) * (ln - 2) // 2)
            total += 20 + (16 if ln < L else 0)
    return total + 30


def _bg_flops_sparse(n, right_leaves, final_leaf):
    L = n - 1
    total = 0
    for ln in range(2, L + 1):
        for a in range(0, L - ln + 1):
            b = a + ln - 1
            for i in range(a, b):
                ll, lr = i == a, right_leaves and i + 1 == b
                d = 16 if (ll and lr) else (18 if (ll or lr) else 30)
                jlkr = 8 if ll else 14
                krjl = 8 if lr else 14
                ax_r = 20 if lr else 32
                ax_l = 20 if ll else 32
                total += d + jlkr + krjl + 4 + ax_r + ax_l + 4 + 16 + 2
                total += (2 if i > a else 0) + (2 if b > i + 1 else 0)
                for j in range(i + 1, b):  # triples ([a..i], [i+1..j], [j+1..b])
                    la, lc = i == a, right_leaves and j + 1 == b
                    total += (16 if (la and lc) else (18 if (la or lc) else 30)) + (20 if j == i + 1 else 32)
            total += 20 + (16 if ln < L else 0)
    return total + (18 if final_leaf else 30)


def bg_flops_leaf(n):
    """bg_flops for the register forms (TESS_K2_REG, _REG_HI, _REG_HI4, _REG_HI_PF,
    _REG_TMA, _REG_TMA_HI; tess_bg.cuh bg_amplitude), which leave out the products
    with the exact zeros of a single leg's polarisation vector (eps^0 and
    Im eps^3): complex dot with one leaf 18 (two leaves 16) instead of 30, a
    leaf's dot with a momentum 8 instead of 14, a multiply-add of a leaf 20
    instead of 32, the final contraction 18."""
    return _bg_flops_sparse(n, True, True)


def bg_flops_wave_unrolled(n):
    """bg_flops for TESS_K2_WAVE2U (every step's code unrolled), which also
    leaves out the zeros of single-leg right and last parts."""
    return _bg_flops_sparse(n, True, False)


def bg_flops_wave(n):
    """bg_flops for the rolled scalar wavefront forms (TESS_K2_WAVE, _WAVE2,
    _WAVE2L; tess_wave.cuh bg_wave, bg_wave_lean), which leave out the zero products where the left
    part of a split, or the first or middle part of a triple, is a single leg
    (the compile-time cases of their step code)."""
    return _bg_flops_sparse(n, False, False)


REGISTER_FORMS = (0, 4, 5, 6, 19, 20, 24)  # TESS_K2_REG, _REG_HI, _REG_TMA, _REG_TMA_HI, _REG_HI4, _REG_HI_PF, _FUSED
WAVE_FORMS = (13, 14, 18)  # TESS_K2_WAVE, _WAVE2, _WAVE2L


def bg_flops_real_leaf(n):
    """bg_flops_real for the real-current register forms (TESS_K2_REAL,
    _REAL_HI; tess_bg.cuh bg_amplitude_real), which leave out the time
    component (exactly zero) of single-leg polarisation vectors: a dot with a
    leaf 5 instead of 7, a multiply-add of a leaf 6 instead of 8, the final
    contraction 5."""
    L = n - 1
    total = 0
    for ln in range(2, L + 1):
        for a in range(0, L - ln + 1):
            b = a + ln - 1
            for i in range(a, b):
                ll, lr = i == a, i + 1 == b
                d = 5 if (ll or lr) else 7
                cr = (5 if ll else 7) + 1
                cl = (5 if lr else 7) + 1
                total += d + cr + cl + (6 if lr else 8) + (6 if ll else 8) + 8 + 4 + 1
                total += (1 if i > a else 0) + (1 if b > i + 1 else 0)
                for j in range(i + 1, b):
                    total += (5 if (i == a or j + 1 == b) else 7) + (6 if j == i + 1 else 8)
            total += 12 + (12 if ln < L else 0)
    return total + 5


def flops_per_event(n, variant, random_pol=False, precision=None):
    """FLOPs of one amplitude as the given amplitude variant evaluates it
    (variant -1: the exact-sum mode's fused kernel, whose recursion is the
    register form for FP32 up to n = 7 and FP64 up to n = 5, else the loop
    form; pass the process's precision)."""
    if variant == -1 and not random_pol:
        reg = n <= 7 if precision in (TESS_FP32_CURRENTS, TESS_FP32_DS) else n <= 5
        return bg_flops_leaf(n) if reg else bg_flops(n)
    if random_pol and variant in (9, 10):  # TESS_K2_REAL, _REAL_HI
        return bg_flops_real_leaf(n)
    if random_pol and variant == 11:  # TESS_K2_ROWS_REAL
        return bg_flops_real(n)
    # the complex-current forms run on real vectors as on helicity vectors
    if variant in REGISTER_FORMS:
        return bg_flops_leaf(n)
    if variant == 15:  # TESS_K2_WAVE2U
        return bg_flops_wave_unrolled(n)
    return bg_flops_wave(n) if variant in WAVE_FORMS else bg_flops(n)


def bg_flops_real(n):
    """The same count for the real-current recursion (random real
    polarisations, tess_bg.cuh bg_amplitude_real): per split 52 (+1 for each
    S term of a multi-leg side), per four-vertex triple 15, per set 12 plus 12
    when propagated, and the final contraction 7."""
    L = n - 1
    total = 0
    for ln in range(2, L + 1):
        for a in range(0, L - ln + 1):
            b = a + ln - 1
            for i in range(a, b):
                total += 52 + (1 if i > a else 0) + (1 if b > i + 1 else 0)
            total += 15 * ((ln - 1) * (ln - 2) // 2)
            total += 12 + (12 if ln < L else 0)
    return total + 7


def splits_and_triples(n):
    L = n - 1
    return math.comb(L + 1, 3), math.comb(L + 1, 4)
