"""FP64 CPU oracle for the gg -> (n-2) gluon leading-colour generator.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (``paper_1002_3446_gb300``) never imports it and has no CPU fallback.

The arithmetic lives in ``tess_oracle.c`` (plain C99, double precision);
this module only builds it with gcc and marshals arguments through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tess_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libtess_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class Process(ctypes.Structure):
    """Mirror of ``orc_process`` in tess_oracle.c."""
    _fields_ = [
        ("n", ctypes.c_int),
        ("hel_mode", ctypes.c_int),
        ("sqrt_s", ctypes.c_double),
        ("pt_min", ctypes.c_double),
        ("eta_max", ctypes.c_double),
        ("dr_min", ctypes.c_double),
        ("alphas_mz", ctypes.c_double),
        ("mz", ctypes.c_double),
        ("nf", ctypes.c_int),
        ("hist_obs", ctypes.c_int),
        ("mu_r_factor", ctypes.c_double),
        ("hist_bins", ctypes.c_int),
        ("grid", ctypes.c_int),
        ("hist_lo", ctypes.c_double),
        ("hist_hi", ctypes.c_double),
    ]


def process(n, hel_mode=1, sqrt_s=14000.0, pt_min=20.0, eta_max=2.5, dr_min=0.4, alphas_mz=0.118,
            mz=91.19, nf=5, mu_r_factor=0.5, hist_obs=0, hist_bins=50, hist_lo=20.0, hist_hi=1020.0, grid=0):
    return Process(n=n, hel_mode=hel_mode, sqrt_s=sqrt_s, pt_min=pt_min, eta_max=eta_max, dr_min=dr_min,
                   alphas_mz=alphas_mz, mz=mz, nf=nf, hist_obs=hist_obs, mu_r_factor=mu_r_factor,
                   hist_bins=hist_bins, grid=grid, hist_lo=hist_lo, hist_hi=hist_hi)


_D = ctypes.POINTER(ctypes.c_double)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_I = ctypes.POINTER(ctypes.c_int)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            h = ctypes.CDLL(build())
            h.orc_philox4x32_10.argtypes = [_U32, _U32, _U32]
            h.orc_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]
            h.orc_uniform.restype = ctypes.c_double
            h.orc_n_uniforms.argtypes = [ctypes.c_int]
            h.orc_n_uniforms_mode.argtypes = [ctypes.c_int, ctypes.c_int]
            h.orc_polvec_real.argtypes = [_D, ctypes.c_double, _D]
            h.orc_grid_pdf.argtypes = [ctypes.POINTER(Process), ctypes.c_float]
            h.orc_grid_pdf.restype = ctypes.c_float
            h.orc_grid_alphas.argtypes = [ctypes.POINTER(Process), ctypes.c_float]
            h.orc_grid_alphas.restype = ctypes.c_float
            h.orc_xg.argtypes = [ctypes.c_double]
            h.orc_xg.restype = ctypes.c_double
            h.orc_rambo.argtypes = [ctypes.c_int, ctypes.c_double, _D, _D]
            h.orc_rambo_weight.argtypes = [ctypes.c_int, ctypes.c_double]
            h.orc_rambo_weight.restype = ctypes.c_double
            h.orc_cuts.argtypes = [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, _D, _D, _D]
            h.orc_alphas.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int]
            h.orc_alphas.restype = ctypes.c_double
            h.orc_polvec.argtypes = [_D, ctypes.c_int, _D]
            h.orc_amp.argtypes = [ctypes.c_int, _I, _D, _D, ctypes.c_int, _D]
            h.orc_event_record.argtypes = [ctypes.POINTER(Process), ctypes.c_uint64, ctypes.c_uint64, _D]
            h.orc_event_record_u.argtypes = [ctypes.POINTER(Process), _D, _D]
            h.orc_generate.argtypes = [ctypes.POINTER(Process), ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_int, _D, _D, _U8, _D, _D, _D, _D, _D]
            h.orc_hist_bin.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double]
            h.orc_compensated_sum.argtypes = [_D, ctypes.c_uint64]
            h.orc_compensated_sum.restype = ctypes.c_double
            _lib = h
        return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


# ---------------------------------------------------------------- wrappers
def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def uniform(seed, ev, j):
    return lib().orc_uniform(seed, ev, j)


def n_uniforms(n, hel_mode=1):
    return lib().orc_n_uniforms_mode(n, hel_mode)


def xg(x):
    return lib().orc_xg(x)


def rambo(m, sqrt_shat, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    p = np.zeros((m, 4))
    lib().orc_rambo(m, sqrt_shat, _dp(u), _dp(p))
    return p


def rambo_weight(m, shat):
    return lib().orc_rambo_weight(m, shat)


def cuts(p, y, pt_min, eta_max, dr_min):
    p = np.ascontiguousarray(p, dtype=np.float64)
    ht, pl, rm = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    ok = lib().orc_cuts(p.shape[0], _dp(p), y, pt_min, eta_max, dr_min, ctypes.byref(ht), ctypes.byref(pl),
                        ctypes.byref(rm))
    return bool(ok), ht.value, pl.value, rm.value


def alphas(mu, alphas_mz=0.118, mz=91.19, nf=5):
    return lib().orc_alphas(mu, alphas_mz, mz, nf)


def polvec(p, h):
    p = np.ascontiguousarray(p, dtype=np.float64)
    e = np.zeros(8)
    lib().orc_polvec(_dp(p), int(h), _dp(e))
    return e[0::2] + 1j * e[1::2]


def grid_pdf(proc, u):
    """Grid-mode x g(x) at the float draw u (interpolated table)."""
    return lib().orc_grid_pdf(ctypes.byref(proc), float(u))


def grid_alphas(proc, v):
    """Grid-mode alpha_s at v = ln mu^2 (float)."""
    return lib().orc_grid_alphas(ctypes.byref(proc), float(v))


def polvec_real(p, phi):
    """Random-polarisation vector cos(phi) e1 + sin(phi) e2 of momentum p (real)."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    e = np.zeros(8)
    lib().orc_polvec_real(_dp(p), float(phi), _dp(e))
    return e[0::2] + 1j * e[1::2]


def amp(order, k, eps, form=0):
    """Colour-ordered amplitude m(order) in the paper's normalisation.

    k: (n,4) all-outgoing momenta; eps: (n,4) complex polarisations."""
    k = np.ascontiguousarray(k, dtype=np.float64)
    n = k.shape[0]
    e = np.zeros((n, 8))
    e[:, 0::2] = np.real(eps)
    e[:, 1::2] = np.imag(eps)
    o = (ctypes.c_int * n)(*[int(x) for x in order])
    out = np.zeros(2)
    lib().orc_amp(n, o, _dp(k), _dp(e), int(form), _dp(out))
    return complex(out[0], out[1])


EVENT_FIELDS = ["x1", "x2", "shat", "y", "alphas", "ht", "ptlead", "rmin", "me2", "weight", "pdf", "phi", "pass",
                "hel_bits"]


def event(proc, seed, ev):
    rec = np.zeros(14 + proc.n + 4 * proc.n)
    rc = lib().orc_event_record(ctypes.byref(proc), seed, ev, _dp(rec))
    if rc:
        raise ValueError("oracle rejected the process")
    d = {f: rec[i] for i, f in enumerate(EVENT_FIELDS)}
    d["pass"] = bool(rec[12])
    d["hel_bits"] = int(rec[13])
    d["perm"] = rec[14:14 + proc.n].astype(int)
    d["k"] = rec[14 + proc.n:].reshape(proc.n, 4).copy()
    return d


def event_u(proc, u):
    """Event from caller-given uniforms (layout as the counter-based draws)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    assert u.size >= n_uniforms(proc.n, proc.hel_mode)
    rec = np.zeros(14 + proc.n + 4 * proc.n)
    if lib().orc_event_record_u(ctypes.byref(proc), _dp(u), _dp(rec)):
        raise ValueError("oracle rejected the process")
    d = {f: rec[i] for i, f in enumerate(EVENT_FIELDS)}
    d["pass"] = bool(rec[12])
    d["hel_bits"] = int(rec[13])
    d["perm"] = rec[14:14 + proc.n].astype(int)
    d["k"] = rec[14 + proc.n:].reshape(proc.n, 4).copy()
    return d


def ulp_sensitivity(proc, seed, ev, trials=6):
    """Largest relative change of the oracle's |A|^2 and weight for event ev
    when each x, Rambo (and polarisation-angle) uniform moves by at most one
    ulp: the difference a
    one-ulp discrepancy in a transcendental function can cause downstream.
    Events near a zero of the amplitude have large values."""
    rng = np.random.default_rng(ev & 0xFFFFFFFF)
    u = uniforms(proc, seed, ev)
    base = event_u(proc, u)
    m = proc.n - 2
    js = list(range(2 + 4 * m))
    if proc.hel_mode == 2:  # and the polarisation angles
        js += list(range(n_uniforms(proc.n, 1), n_uniforms(proc.n, 2)))
    worst = 0.0
    for _ in range(trials):
        up = u.copy()
        for j in js:
            r = rng.integers(3)
            if r:
                up[j] = np.nextafter(up[j], 0.0 if r == 1 else 1.0)
        e = event_u(proc, up)
        if e["pass"] != base["pass"] or base["me2"] == 0:
            continue
        worst = max(worst, abs(e["me2"] - base["me2"]) / abs(base["me2"]))
        if base["weight"] > 0:
            worst = max(worst, abs(e["weight"] - base["weight"]) / base["weight"])
    return worst


def uniforms(proc_or_n, seed, ev):
    if isinstance(proc_or_n, int):
        n, mode = proc_or_n, 1
    else:
        n, mode = proc_or_n.n, proc_or_n.hel_mode
    return np.array([uniform(seed, ev, j) for j in range(n_uniforms(n, mode))])


def generate(proc, seed, first, n_events, threads=None, per_event=True, hist=True):
    """Run the oracle over events [first, first+n_events).  Returns a dict."""
    threads = threads or os.cpu_count() or 1
    out = {}
    ptrs = []
    for name in ("weight", "me2", "ht", "ptlead", "rmin"):
        if per_event:
            out[name] = np.zeros(n_events)
            ptrs.append(_dp(out[name]))
        else:
            ptrs.append(None)
    if per_event:
        out["pass"] = np.zeros(n_events, dtype=np.uint8)
        pp = out["pass"].ctypes.data_as(_U8)
    else:
        pp = None
    acc = np.zeros(4)
    h = np.zeros(2 * (proc.hist_bins + 2)) if hist else None
    rc = lib().orc_generate(ctypes.byref(proc), seed, first, n_events, threads, ptrs[0], ptrs[1], pp, ptrs[2],
                            ptrs[3], ptrs[4], _dp(acc), _dp(h) if hist else None)
    if rc:
        raise ValueError("oracle generate failed")
    out["acc"] = acc
    if hist:
        nb = proc.hist_bins
        out["hist_w"] = h[:nb + 2]
        out["hist_w2"] = h[nb + 2:]
    out["threads"] = threads
    return out


def sigma(acc):
    """Cross section and its Monte Carlo error (pb) from (sum w, sum w^2, n_pass, n_gen)."""
    sw, sw2, _, n = acc
    mean = sw / n
    var = (sw2 / n - mean * mean) / max(n - 1, 1)
    return mean, float(np.sqrt(max(var, 0.0)))


def compensated_sum(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_compensated_sum(_dp(x), x.size)
