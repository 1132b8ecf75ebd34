#!/usr/bin/env python3
"""Benchmark of the gg -> (n-2) gluon event generator on GB300.

A step = one tess_generate call over the whole workload: counter RNG ->
Rambo -> luminosity, alpha_s, cuts, observables -> polarisations ->
Berends-Giele amplitude -> weight -> cross-section/histogram accumulation,
writing per-event weight, |A|^2 estimator and pass flag.

Default workload "gg4g": gg -> 4 gluons (6-point), 2^24 events per GPU,
sampled helicity and colour ordering, FP32 currents (FP64 plain form
measured alongside).  Multi-GPU: each rank generates its own disjoint event
range (weak scaling); the only exchange is the sum of the accumulators.

``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

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
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (n, events per GPU, pt_min, helicity mode, precision, hist (obs, bins, lo, hi))
    "gg4g": dict(n=6, n_events=1 << 24, pt_min=20.0, hel="sample", precision="ds", hist=None),
    "gg2g": dict(n=4, n_events=1 << 20, pt_min=20.0, hel="sum", precision="fp64", hist=(0, 50, 20.0, 1020.0)),
    "gg8g": dict(n=10, n_events=1 << 26, pt_min=30.0, hel="sample", precision="ds", hist=(1, 40, 200.0, 3000.0)),
}
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12   # 80.5, from unit counts and clock
FP64_PEAK_TFLOPS = 1.25                                                     # GB300 FP64 (vendor figure)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tess", choices=["tess", "reference"])
    ap.add_argument("--workload", default="gg4g", choices=sorted(WORKLOADS))
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison measurement")
    ap.add_argument("--no-per-n", action="store_true", help="skip the per-multiplicity sweep")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the gg->2g (2^20, FP64 exact sum) and gg->8g (2^26) configuration legs")
    ap.add_argument("--no-peaks", action="store_true", help="skip the FMA peak probes (nominal peak instead)")
    ap.add_argument("--events", type=int, default=0, help="override events per GPU (small cases for profiling)")
    ap.add_argument("--chunk-mb", type=int, default=0,
                    help="chunk size of the generation pipeline in MiB (tess_set_chunk_bytes; 0: the library default)")
    ap.add_argument("--no-batched", action="store_true", help="skip the mixed-multiplicity batched measurement")
    ap.add_argument("--no-grad", action="store_true", help="skip the gradient measurement")
    ap.add_argument("--grad-only", action="store_true",
                    help="time only the gradient path (gg -> 6 gluons; --events overrides 2^22) and print its line")
    ap.add_argument("--no-autotune", action="store_true", help="time the built-in default amplitude variant")
    ap.add_argument("--no-random-pol", action="store_true", help="skip the random-polarisation measurement")
    ap.add_argument("--no-cut-first", action="store_true", help="skip the cut-first measurements")
    ap.add_argument("--no-pdf-grid", action="store_true",
                    help="skip the measurement with tabulated PDF and alpha_s (TESS_FLAG_PDF_GRID)")
    ap.add_argument("--cut-first", action="store_true",
                    help="the whole line with TESS_FLAG_CUT_FIRST (amplitudes only for events passing the cuts)")
    ap.add_argument("--pol", default="helicity", choices=["helicity", "random"],
                    help="sampled helicities (default) or the paper's random real polarisations (TESS_POL_RANDOM)")
    ap.add_argument("--variant", default="", help="FORM,SCHEDULE: use this amplitude variant and chunk schedule "
                                                 "instead of autotuning (reproducible profiling)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples (every 20 ms, each with its host time) while the
    block runs; summary(window) keeps those inside the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.rows = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t_end = time.monotonic() + 5.0  # sampling live before the timed region starts
            while not self.rows and self.proc.poll() is None and time.monotonic() < t_end:
                time.sleep(0.01)
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append((time.monotonic(), parts))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self, window=None):
        rows = [r for t, r in self.rows if window is None or window[0] <= t <= window[1]]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ tess arm
def make_proc(tess, wl, precision=None, random_pol=False):
    prec = precision or wl["precision"]
    mode = tess.TESS_HEL_SUM if wl["hel"] == "sum" else (tess.TESS_POL_RANDOM if random_pol else tess.TESS_HEL_SAMPLE)
    kw = dict(precision={"fp32": tess.TESS_FP32_CURRENTS, "ds": tess.TESS_FP32_DS, "fp64": tess.TESS_FP64}[prec],
              helicity_mode=mode, pt_min=wl["pt_min"])
    if wl["hist"]:
        obs, nb, lo, hi = wl["hist"]
        kw.update(hist_observable=obs, hist_bins=nb, hist_lo=lo, hist_hi=hi)
    return tess.process(wl["n"], **kw)


def precision_error(torch, r, r64):
    """Per-event relative difference |w - w64| / |w64| of an FP32-current run
    against the FP64 run of the same events (the FP64 form agrees with the
    oracle to 1e-10 per event): median, 99th percentile and maximum over the
    events both pass; events whose FP64 |A|^2 is below 1e-16 of the median
    (helicity configurations whose amplitude vanishes, where both forms return
    rounding noise) are counted, not compared; cut decisions that differ are
    counted (the FP32 forms take them on FP32 momenta).  The tail (above_1e_2)
    is ill-conditioned events: the parity tests bound each event's FP32 error
    by 16 times the change of its FP64 result when its inputs move by an FP32
    rounding."""
    p, p64 = r.t["pass"].bool(), r64.t["pass"].bool()
    both = p & p64
    m64 = r64.t["me2"][both].abs()
    med = float(m64.median()) if m64.numel() else 0.0
    live = m64 > 1e-16 * med
    w, w64 = r.t["weight"][both][live], r64.t["weight"][both][live]
    rel = ((w - w64).abs() / w64.abs()).double()
    out = {"events": int(r.n_events), "compared": int(rel.numel()), "vanishing": int((~live).sum()),
           "cut_flips": int((p != p64).sum())}
    if rel.numel():
        step = max(1, rel.numel() // (1 << 23))  # torch.quantile's input limit
        out.update(median=float(rel.median()), p99=float(torch.quantile(rel[::step], 0.99)), max=float(rel.max()),
                   above_1e_2=int((rel > 1e-2).sum()))
    return out


def time_steps(torch, run, seed, first, steps, warmup, flush, window=None):
    """Device times (ms) of `steps` calls after `warmup` untimed ones; window, if
    given, receives the host times that bracket the timed calls."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        run.reset()
        run.generate(seed, first)
    torch.cuda.synchronize()
    t0 = time.monotonic()
    evs = []
    for _ in range(steps):
        flush.fill_(1.0)  # evict L2 (buffer larger than the 129 MB L2); not timed
        run.reset()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run.generate(seed, first)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    if window is not None:
        window[:] = [t0, time.monotonic()]
    return [a.elapsed_time(b) for a, b in evs]


def measure_peaks(torch, tess, ctx, gpu_id):
    """FMA peaks of this GPU (tess_peak_flops) with the SM clock sampled while
    they run: the roofline denominators of this run."""
    out = {}
    with ClockSampler(gpu_id) as clk:
        t0 = time.monotonic()
        for name, kind in (("fp32", tess.TESS_PEAK_FP32), ("fp32x2", tess.TESS_PEAK_FP32X2),
                           ("fp64", tess.TESS_PEAK_FP64)):
            out[name] = tess.tess_peak_flops(ctx, kind, reps=20)
        t1 = time.monotonic()
    out["clocks"] = clk.summary([t0, t1])
    out["nominal_fp32"] = FP32_PEAK_TFLOPS
    return out


def peak_at(peaks, key, sm_mhz):
    """Measured peak `key`, rescaled from the probe's median SM clock to sm_mhz."""
    v = peaks[key]
    c0 = peaks["clocks"].get("sm_mhz")
    if c0 and sm_mhz:
        v *= sm_mhz / c0
    return v


def sig(x, d=4):
    """x rounded to d significant digits (compact JSON)."""
    if x is None:
        return None
    if isinstance(x, (list, tuple)):
        return [sig(v, d) for v in x]
    if isinstance(x, dict):
        return {k: sig(v, d) for k, v in x.items()}
    if isinstance(x, bool) or isinstance(x, int):
        return x
    try:
        return float(f"{x:.{d}g}")
    except (TypeError, ValueError):
        return x


def amp_kernel_time(torch, tess, ctx, proc, run, seed, first, flush, steps):
    """Device time per step (ms) of the amplitude kernel (or the fused kernel
    of the exact-sum mode), from the library's CUDA events around each launch,
    with the kernels run serially (an overlapped schedule is switched to its
    serial counterpart with the same variant for this measurement)."""
    N = run.n_events
    plan = tess.tess_plan_info(ctx, proc, N)
    serial_of = {tess.TESS_SCHED_OVERLAP: tess.TESS_SCHED_SERIAL,
                 tess.TESS_SCHED_OVERLAP_TILES: tess.TESS_SCHED_SERIAL_TILES}
    if plan["schedule"] in serial_of:
        tess.tess_select_variant(ctx, proc, plan["variant"], serial_of[plan["schedule"]])
    tess.tess_stage_timing(ctx, 1)
    tess.tess_stage_times(ctx)
    for _ in range(steps):
        flush.fill_(1.0)
        run.reset()
        run.generate(seed, first)
    st = tess.tess_stage_times(ctx)
    tess.tess_stage_timing(ctx, 0)
    if plan["schedule"] in serial_of:
        tess.tess_select_variant(ctx, proc, plan["variant"], plan["schedule"])
    ms, launches = st["amplitude"]
    if launches == 0:
        ms, launches = st["fused"]
    return ms / steps, launches // steps, plan, st


def bench_config(torch, tess, ctx, name, flush, steps, peaks, sm_mhz, autotune=True, with_cpu=True,
                 forms=("ds", "fp32", "fp64"), fp64_events=None):
    """One workload of the numerical study at its stated size: events/s of
    each precision form, sigma +- MC error, the amplitude kernel's roofline
    (FLOPs counted from the kernel's inner loop x events / its serial device
    time, against the FMA peak measured in this run), the FP32 forms' per-event
    error against the FP64 form on the same events, and the oracle on the
    host cores."""
    wl = dict(WORKLOADS[name])
    N, n = wl["n_events"], wl["n"]
    res = {"workload": workload_config(name, wl, N)["workload"]}
    runs = {}
    for form in forms:
        if wl["precision"] == "fp64" and form != "fp64":
            continue
        ne = N if form != "fp64" or wl["precision"] == "fp64" else (fp64_events or N >> 3)
        proc = make_proc(tess, wl, form)
        run = tess.Run(ctx, proc, ne, per_event=("weight", "me2", "pass"))
        if autotune and wl["hel"] == "sample":
            tess.tess_autotune(ctx, proc, min(ne, 1 << 25), None, run.workspace, outputs=run.outputs)
        ms = statistics.mean(time_steps(torch, run, 1, 0, steps, 2, flush))
        amp_ms, amp_launches, plan, _ = amp_kernel_time(torch, tess, ctx, proc, run, 1, 0, flush, steps)
        # the exact sum evaluates (n-1)! orderings x 2^(n-1) helicity labellings per event (flipping every
        # label leaves |m| unchanged, so leg 0 keeps label 0 and the sum is doubled)
        evals = ne * (math.factorial(n - 1) * 2 ** (n - 1) if wl["hel"] == "sum" else 1)
        fl = tess.flops_per_event(n, plan["variant"], precision=proc.precision)  # as the timed variant evaluates it
        achieved = fl * evals / (amp_ms * 1e-3) / 1e12
        pk = peak_at(peaks, "fp64" if form == "fp64" else "fp32", sm_mhz)
        sg = run.result()
        entry = {"events": ne, "value": ne / (ms * 1e-3), "ms_per_step": ms, "sigma_pb": [sg[0], sg[1]],
                 "n_pass": sg[2],
                 "roofline": {"bound": "alu", "achieved": achieved, "peak": pk,
                              "peak_kind": "measured " + ("FP64" if form == "fp64" else "FP32") + " FMA rate",
                              "unit": "TFLOP/s", "frac": achieved / pk, "flops_per_amplitude": fl,
                              "amplitudes_per_event": evals // ne, "kernel_ms_per_step": amp_ms,
                              "launches_per_step": amp_launches, "variant_schedule": [plan["variant"],
                                                                                      plan["schedule"]],
                              "traffic": read_traffic(name if form != "fp64" else name + "_fp64", plan["variant"],
                                                      min(ne, plan_cap(tess, ctx, proc, ne)))}}
        if wl["hist"] and form == forms[0]:
            hw, hw2 = run.histograms()
            entry["hist_sumw"] = [float(x) for x in hw]
        res[form] = entry
        runs[form] = run
    if "fp64" in runs and wl["precision"] != "fp64":
        r64 = runs["fp64"]
        ne = r64.n_events
        for form in forms:
            if form == "fp64":
                continue
            rf = tess.Run(ctx, make_proc(tess, wl, form), ne, per_event=("weight", "me2", "pass"))
            rf.reset()
            rf.generate(1, 0)
            torch.cuda.synchronize()
            res[form]["error_vs_fp64"] = precision_error(torch, rf, r64)
            del rf
    del runs
    if with_cpu:
        res["cpu_baseline"] = cpu_baseline(wl, budget_s=10.0)
    return res


def compact_config(res):
    """The few numbers of a bench_config result that the summary keeps."""
    out = {}
    for form in ("ds", "fp32", "fp64"):
        if form in res:
            e = res[form]
            r = e["roofline"]
            out[form] = {"ev_s": sig(e["value"]), "tflops": sig(r["achieved"], 3), "frac": sig(r["frac"], 3)}
            if "error_vs_fp64" in e:
                er = e["error_vs_fp64"]
                out[form]["err"] = sig({"med": er.get("median"), "p99": er.get("p99"), "max": er.get("max")}, 2)
    first = next(f for f in ("ds", "fp32", "fp64") if f in res)
    out["sigma"] = sig(res[first]["sigma_pb"], 5)
    if "cpu_baseline" in res:
        out["cpu_ev_s"] = sig(res["cpu_baseline"]["value"], 3)
        out["cpu_cores"] = res["cpu_baseline"]["cores"]
    return out


def summary_of(line, configs, peaks):
    """Compact restatement of the line's key figures, printed last so that a
    record keeping only the end of the line still holds them: the measured
    peaks, each configuration's events/s per precision form with its
    amplitude-kernel TFLOP/s and fraction of the measured peak, the FP32
    forms' error against FP64, sigma, the batched comparison and the oracle."""
    out = {}
    if peaks:
        out["peak_tflops"] = sig({"fp32": peaks["fp32"], "fp32x2": peaks["fp32x2"], "fp64": peaks["fp64"],
                                  "sm_mhz": peaks["clocks"].get("sm_mhz")}, 4)
    r = line["roofline"]
    c2 = {"ds": {"ev_s": sig(line["value"]), "tflops": sig(r["achieved"], 3), "frac": sig(r["frac"], 3)},
          "e2e_ev_s": sig(line["e2e"]["value"])}
    if "fp32_native_fp64_steps" in line:
        c2["fp32"] = {"ev_s": sig(line["fp32_native_fp64_steps"]["value"])}
    if "fp64" in line:
        f = line["fp64"]
        c2["fp64"] = {"ev_s": sig(f["value"]), "tflops": sig(f["achieved_tflops"], 3),
                      "frac": sig(f["achieved_tflops"] / f["peak_tflops"], 3)}
        er = next((v for k, v in f.items() if k.startswith("error_of_")), None)
        if er:
            c2["ds"]["err"] = sig({"med": er.get("median"), "p99": er.get("p99"), "max": er.get("max")}, 2)
    if line.get("cpu_baseline"):
        c2["cpu_ev_s"] = sig(line["cpu_baseline"]["value"], 3)
    if "C1_gg2g" in configs:
        out["C1"] = compact_config(configs["C1_gg2g"])
    out["C2"] = c2
    if "C3_gg8g" in configs:
        out["C3"] = compact_config(configs["C3_gg8g"])
    b = line.get("batched_mixed")
    if b:
        out["C4"] = {k: sig(b[k]["value"]) for k in ("plain_9_launches_autotuned", "graph_batched_autotuned",
                                                      "persistent_graph") if k in b}
    g = line.get("gradients_gg6g")
    if g:
        out["C5_grad_ev_s"] = sig(g["value"])
    return out


def run_tess(args):
    import torch
    import paper_1002_3446_gb300 as tess

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = dict(WORKLOADS[args.workload])
    if args.events:
        wl["n_events"] = args.events
    n, N = wl["n"], wl["n_events"]
    rp = args.pol == "random" and wl["hel"] == "sample"
    flops_per_event = tess.bg_flops_real(n) if rp else tess.bg_flops(n)
    ctx = tess.tess_init(local)
    if args.chunk_mb:
        tess.tess_set_chunk_bytes(ctx, args.chunk_mb << 20)
    proc = make_proc(tess, wl, random_pol=rp)
    cf = args.cut_first and wl["hel"] == "sample" and wl["precision"] in ("fp32", "ds")
    if cf:
        proc.flags = tess.TESS_FLAG_CUT_FIRST
    run = tess.Run(ctx, proc, N, per_event=("weight", "me2", "pass"))
    variant = None
    if args.variant:
        form, sched = (int(x) for x in args.variant.split(","))
        tess.tess_select_variant(ctx, proc, form, sched)
    elif not args.no_autotune and wl["hel"] == "sample":
        probe_acc = torch.zeros(tess.TESS_ACC_LEN, dtype=torch.float64, device="cuda")
        # tuned on the workload itself (candidates within a few per cent of each
        # other change order between a 2^22-event probe and the full size)
        variant = tess.tess_autotune(ctx, proc, min(N, 1 << 25), probe_acc, run.workspace, outputs=run.outputs)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")  # 256 MB > L2
    from paper_1002_3446_gb300 import dist as tdist
    first, _ = tdist.event_range(rank, ws, N)
    seed = 1

    def barrier():
        if dist:
            dist.barrier()

    try:
        gpu_id = torch.cuda.get_device_properties(local).uuid
        gpu_id = "GPU-" + str(gpu_id) if not str(gpu_id).startswith("GPU-") else str(gpu_id)
    except Exception:
        gpu_id = str(local)

    peaks = None if args.no_peaks else measure_peaks(torch, tess, ctx, gpu_id)

    # ---- headline: device time of K steps
    barrier()
    torch.cuda.synchronize()
    timed_window = []
    with ClockSampler(gpu_id) as clk:
        step_ms = time_steps(torch, run, seed, first, args.steps, args.warmup, flush, timed_window)
    torch.cuda.synchronize()
    barrier()
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = ws * N / (ms_per_step * 1e-3)
    sigma = run.result()
    acc = run.acc.clone()
    n_pass_local = int(acc[2].item())  # passing events of this rank's last step

    # ---- per-stage device time (library-recorded CUDA events on the launch stream).
    # Under an overlapped schedule the two kernels share the SMs, so the stages
    # are timed with the same kernel variants run serially (each kernel alone).
    plan = tess.tess_plan_info(ctx, proc, N)
    flops_per_event = tess.flops_per_event(n, plan["variant"], rp, precision=proc.precision)  # as the chosen variant evaluates it
    serial_of = {tess.TESS_SCHED_OVERLAP: tess.TESS_SCHED_SERIAL,
                 tess.TESS_SCHED_OVERLAP_TILES: tess.TESS_SCHED_SERIAL_TILES}
    if plan["schedule"] in serial_of:
        tess.tess_select_variant(ctx, proc, plan["variant"], serial_of[plan["schedule"]])
    tess.tess_stage_timing(ctx, 1)
    tess.tess_stage_times(ctx)
    for _ in range(args.steps):
        flush.fill_(1.0)
        run.reset()
        run.generate(seed, first)
    stages = tess.tess_stage_times(ctx)
    tess.tess_stage_timing(ctx, 0)
    if plan["schedule"] in serial_of:
        tess.tess_select_variant(ctx, proc, plan["variant"], plan["schedule"])
    if dist:
        dist.all_reduce(acc, op=dist.ReduceOp.SUM)

    # ---- end to end: public API with host buffers.  The per-event weights,
    # |m|^2 and flags land in pinned host memory (the kernels store there directly over
    # NVLink-C2C), sigma is read back by tess_result; same variant and schedule.
    host_run = tess.Run(ctx, proc, N, per_event=("weight", "me2", "pass"), host_per_event=True)
    for _ in range(2):
        host_run.reset()
        host_run.generate(seed, first)
        host_run.result()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        host_run.reset()
        host_run.generate(seed, first)
        host_run.result()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    barrier()
    if dist:
        t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())

    # ---- FP64 plain form of the same workload, and the per-n sweep
    extra = {}
    if wl["precision"] == "ds" and rank == 0:
        p32 = make_proc(tess, wl, "fp32", random_pol=rp)
        r32 = tess.Run(ctx, p32, N, per_event=("weight", "me2", "pass"))
        ms = time_steps(torch, r32, seed, first, max(2, args.steps // 2), 2, flush)
        extra["fp32_native_fp64_steps"] = {
            "value": N / (statistics.mean(ms) * 1e-3), "ms_per_step": statistics.mean(ms),
            "note": "TESS_FP32_CURRENTS: Rambo boost/rescale and polarisation Gram products in native FP64"}
        del r32
    if not args.no_fp64 and wl["precision"] in ("fp32", "ds") and rank == 0:
        p64 = make_proc(tess, wl, "fp64", random_pol=rp)
        n64 = N >> 3
        r64 = tess.Run(ctx, p64, n64, per_event=("weight", "me2", "pass"))
        ms = time_steps(torch, r64, seed, first, max(1, args.steps // 2), 1, flush)
        extra["fp64"] = {"value": n64 / (statistics.mean(ms) * 1e-3), "events": n64,
                         "ms_per_step": statistics.mean(ms),
                         "achieved_tflops": tess.bg_flops(n) * n64 / (statistics.mean(ms) * 1e-3) / 1e12,
                         "peak_tflops": peaks["fp64"] if peaks else FP64_PEAK_TFLOPS}
        # the main form's per-event error against the FP64 form on the same events
        rf = tess.Run(ctx, proc, n64, per_event=("weight", "me2", "pass"))
        rf.reset()
        rf.generate(seed, first)
        torch.cuda.synchronize()
        extra["fp64"]["error_of_" + wl["precision"]] = precision_error(torch, rf, r64)
        del r64, rf
    if not rp and not cf and not args.no_random_pol and wl["hel"] == "sample" and wl["precision"] in ("fp32", "ds") \
            and rank == 0:
        extra["random_polarisation"] = bench_random_pol(torch, tess, ctx, wl, N, seed, first, flush,
                                                        max(2, args.steps // 2), not args.no_autotune)
    if not rp and not cf and not args.no_cut_first and wl["hel"] == "sample" and wl["precision"] in ("fp32", "ds") \
            and rank == 0:
        extra["cut_first"] = bench_random_pol(torch, tess, ctx, wl, N, seed, first, flush, max(2, args.steps // 2),
                                              not args.no_autotune, random_pol=False,
                                              flags=tess.TESS_FLAG_CUT_FIRST)
        extra["cut_first_random_polarisation"] = bench_random_pol(
            torch, tess, ctx, wl, N, seed, first, flush, max(2, args.steps // 2), not args.no_autotune,
            random_pol=True, flags=tess.TESS_FLAG_CUT_FIRST)
    if not rp and not cf and not args.no_pdf_grid and wl["hel"] == "sample" and wl["precision"] in ("fp32", "ds") \
            and rank == 0:
        extra["pdf_grid"] = bench_random_pol(torch, tess, ctx, wl, N, seed, first, flush, max(2, args.steps // 2),
                                             not args.no_autotune, random_pol=False,
                                             flags=tess.TESS_FLAG_PDF_GRID)
    if not args.no_batched and rank == 0:
        extra["batched_mixed"] = bench_batched(torch, tess, ctx, flush, max(2, args.steps // 2))
    if not args.no_grad and rank == 0:
        extra["gradients_gg6g"] = bench_gradients(torch, tess, ctx, max(2, args.steps // 2))
    main_clocks = clk.summary(timed_window)
    configs = {}
    if not args.no_configs and rank == 0 and not args.events and not rp and not cf and peaks:
        configs["C1_gg2g"] = bench_config(torch, tess, ctx, "gg2g", flush, max(2, args.steps // 4), peaks,
                                          main_clocks.get("sm_mhz"), with_cpu=not args.no_cpu_baseline)
        configs["C3_gg8g"] = bench_config(torch, tess, ctx, "gg8g", flush, max(2, args.steps // 4), peaks,
                                          main_clocks.get("sm_mhz"), autotune=not args.no_autotune,
                                          with_cpu=not args.no_cpu_baseline, fp64_events=1 << 23)
    if not args.no_per_n and rank == 0:
        sweep = {}
        for nn in range(4, 13):
            row = {}
            for prec in ("ds", "fp32", "fp64"):
                w2 = dict(wl, n=nn, pt_min=30.0 if nn >= 10 else 20.0, hel="sample", hist=None)
                pp = make_proc(tess, w2, prec)
                ne = (1 << 16) if prec == "fp64" else (1 << 20)
                rr = tess.Run(ctx, pp, ne, per_event=("weight",))
                if not args.no_autotune:
                    tess.tess_autotune(ctx, pp, ne, None, rr.workspace, outputs=rr.outputs)
                ms = time_steps(torch, rr, seed, 0, 2, 1, flush)
                ev = ne / (min(ms) * 1e-3)
                info = tess.tess_plan_info(ctx, pp, ne)
                row[prec] = {"events_per_s": ev, "tflops": tess.flops_per_event(nn, info["variant"]) * ev / 1e12,
                             "variant_schedule": [info["variant"], info["schedule"]]}
                del rr
            sweep[str(nn)] = row
        extra["per_n"] = sweep

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, budget_s=12.0, random_pol=rp)

    if rank == 0:
        amp_ms, amp_launches = stages["amplitude"]
        if amp_launches == 0:  # exact-sum mode: one fused kernel
            amp_ms, amp_launches = stages["fused"]
        amp_ms_step = amp_ms / args.steps
        evaluated = n_pass_local if cf else N  # amplitudes computed per step (cut-first: passing events)
        if wl["hel"] == "sum":  # every colour ordering and helicity labelling of each event (leg 0's label fixed)
            evaluated = N * math.factorial(n - 1) * 2 ** (n - 1)
        achieved = flops_per_event * evaluated / (amp_ms_step * 1e-3) / 1e12
        tot = sum(v[0] for v in stages.values()) or 1.0
        traffic = read_traffic(args.workload + ("_rp" if rp else "") + ("_cf" if cf else ""), plan["variant"],
                               min(N, plan_cap(tess, ctx, proc, N)))
        kind = "fp64" if wl["precision"] == "fp64" else "fp32"
        nominal = FP64_PEAK_TFLOPS if kind == "fp64" else FP32_PEAK_TFLOPS
        peak = peak_at(peaks, kind, main_clocks.get("sm_mhz")) if peaks else nominal
        line = {
            "metric": workload_metric(wl),
            "value": value,
            "unit": "events/s",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_per_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"fp32": "f32 currents and cuts; f64 Rambo rescale, polarisations, accumulation",
                      "ds": ("f32 currents, cuts and polarisation basis; double-float (2 x f32) Rambo boost and "
                             "rescale; f64 weights and accumulation"),
                      "fp64": "f64"}[wl["precision"]],
            "data": "synthetic (counter-based Philox draws, toy gluon PDF)",
            "config": dict(workload_config(args.workload, wl, N, rp, cf),
                           l2="flushed between timed steps (256 MB write)",
                           chunk_mb=args.chunk_mb or "library default (4096)"),
            "roofline": {"bound": "alu", "kernel": "Berends-Giele amplitude kernel", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                         "peak_source": ((f"measured in this run: {kind.upper()} FMA probe (tess_peak_flops), "
                                          "rescaled to the timed region's median SM clock") if peaks else
                                         "nominal: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"),
                         "peak_nominal": nominal,
                         "frac_of_nominal": achieved / nominal,
                         "flops_per_event": flops_per_event, "ms_per_step": amp_ms_step,
                         "variant": variant,
                         "plan": plan,
                         "launches_per_step": amp_launches // args.steps,
                         "timed": ("CUDA events recorded by the library around each amplitude launch"
                                   + (", kernels run serially (same variants)" if plan["schedule"] in serial_of
                                      else ""))},
            "stage_share": {k: v[0] / tot for k, v in stages.items() if v[1] > 0},
            "e2e": {"value": ws * N / e2e_s, "unit": "events/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": N * 17 + 64,
                    "how": "tess_generate with the per-event weight, |m|^2 and pass arrays in pinned host memory "
                           "(stored by the kernels over NVLink-C2C) + tess_result; the inputs are the seed and "
                           "event range"},
            "gpu_launches": tess.tess_kernel_launches(ctx, proc, N) * args.steps,
            "clocks": main_clocks,
            "sigma_pb": float((acc[0] + acc[4]).item() / (ws * N)),
            "cpu_baseline": cpu,
        }
        line.update(extra)
        line["peaks"] = peaks
        line.update(configs)
        line["summary"] = summary_of(line, configs, peaks)
        print(json.dumps(line), flush=True)
    tess.tess_destroy(ctx)
    if dist:
        dist.destroy_process_group()


def bench_batched(torch, tess, ctx, flush, steps):
    """gg -> 2..10 gluons (n = 4..12) with 2^24 .. 2^16 events, FP32 currents:
    one graph launch of the batched call vs 9 separate tess_generate calls,
    before and after autotuning the amplitude kernel per n."""
    ns = list(range(4, 13))
    counts = [1 << (24 - i) for i in range(9)]
    procs = [tess.process(n, precision=tess.TESS_FP32_DS, pt_min=30.0 if n >= 10 else 20.0) for n in ns]
    runs = [tess.Run(ctx, p, c, per_event=("weight",)) for p, c in zip(procs, counts)]
    ws_bytes = tess.tess_workspace_size_batched(ctx, procs, counts)
    ws = torch.empty((ws_bytes + 7) // 8, dtype=torch.float64, device="cuda")
    outs = [r.outputs for r in runs]
    seeds, firsts = [1] * 9, [0] * 9
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.mean(ts)

    def batched():
        tess.tess_generate_batched(ctx, procs, seeds, firsts, counts, outs, ws)

    def plain():
        for r in runs:
            r.generate(1, 0)

    total = sum(counts)
    res = {"events": total, "n": ns, "events_per_n": counts}
    ms = timed(plain)
    res["plain_9_launches"] = {"value": total / (ms * 1e-3), "ms": ms}
    ms = timed(batched)
    res["graph_batched"] = {"value": total / (ms * 1e-3), "ms": ms}
    acc = torch.zeros(tess.TESS_ACC_LEN, dtype=torch.float64, device="cuda")
    chosen = {}
    for p, r in zip(procs, runs):
        probe = min(r.n_events, 1 << 21)
        tess.tess_autotune(ctx, p, probe, acc, r.workspace, outputs=r.outputs)
        info = tess.tess_plan_info(ctx, p, r.n_events)
        chosen[p.n_gluons] = [info["variant"], info["schedule"]]
    ms = timed(batched)
    res["graph_batched_autotuned"] = {"value": total / (ms * 1e-3), "ms": ms, "variant_schedule": chosen}
    ms = timed(plain)
    res["plain_9_launches_autotuned"] = {"value": total / (ms * 1e-3), "ms": ms}
    # one persistent launch over every multiplicity (atomic work counter), captured in a graph
    pws_bytes = tess.tess_workspace_size_persistent(ctx, procs, counts)
    pws = torch.empty((pws_bytes + 7) // 8, dtype=torch.float64, device="cuda")

    def persistent():
        tess.tess_generate_persistent(ctx, procs, seeds, firsts, counts, outs, pws)

    ms = timed(persistent)
    res["persistent"] = {"value": total / (ms * 1e-3), "ms": ms}
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=cs, capture_error_mode="thread_local"):
        tess.tess_generate_persistent(ctx, procs, seeds, firsts, counts, outs, pws, stream=cs)
    ms = timed(g.replay)
    res["persistent_graph"] = {"value": total / (ms * 1e-3), "ms": ms}
    res["unit"] = "events/s"
    return res


def bench_random_pol(torch, tess, ctx, wl, N, seed, first, flush, steps, autotune, random_pol=True, flags=0):
    """The same workload with the paper's random real polarisations
    (TESS_POL_RANDOM) instead of sampled helicities -- real currents, so the
    real-current amplitude forms apply; FLOPs from bg_flops_real -- and/or
    with process flags (TESS_FLAG_CUT_FIRST: amplitudes only for the events
    that pass the cuts, the amplitude kernel's FLOP rate then counting the
    evaluated events; TESS_FLAG_PDF_GRID: PDF and alpha_s interpolated from
    tables, Sec. 3)."""
    p = make_proc(tess, wl, random_pol=random_pol)
    p.flags = flags
    r = tess.Run(ctx, p, N, per_event=("weight", "me2", "pass"))
    if autotune:
        tess.tess_autotune(ctx, p, min(N, 1 << 22), None, r.workspace, outputs=r.outputs)
    ms = time_steps(torch, r, seed, first, steps, 2, flush)
    info = tess.tess_plan_info(ctx, p, N)
    serial_of = {tess.TESS_SCHED_OVERLAP: tess.TESS_SCHED_SERIAL,
                 tess.TESS_SCHED_OVERLAP_TILES: tess.TESS_SCHED_SERIAL_TILES}
    if info["schedule"] in serial_of:
        tess.tess_select_variant(ctx, p, info["variant"], serial_of[info["schedule"]])
    tess.tess_stage_timing(ctx, 1)
    tess.tess_stage_times(ctx)
    for _ in range(steps):
        flush.fill_(1.0)
        r.reset()
        r.generate(seed, first)
    st = tess.tess_stage_times(ctx)
    tess.tess_stage_timing(ctx, 0)
    tess.tess_select_variant(ctx, p, info["variant"], info["schedule"])
    amp_ms, amp_n = st["amplitude"]
    res_ = r.result()
    fl = tess.flops_per_event(wl["n"], info["variant"], random_pol)
    evaluated = res_[2] if flags & tess.TESS_FLAG_CUT_FIRST else N  # amplitudes computed per step
    res = {"value": N / (statistics.mean(ms) * 1e-3), "unit": "events/s", "ms_per_step": statistics.mean(ms),
           "sigma_pb": res_[:2], "variant_schedule": [info["variant"], info["schedule"]],
           "amplitudes_per_step": evaluated}
    if amp_n:
        amp_step_ms = amp_ms / steps
        res["amplitude_kernel"] = {"tflops": fl * evaluated / (amp_step_ms * 1e-3) / 1e12,
                                   "peak_tflops": FP32_PEAK_TFLOPS, "flops_per_event": fl,
                                   "ms_per_step": amp_step_ms}
    del r
    return res


def bench_gradients(torch, tess, ctx, steps, E=1 << 22):
    """gg -> 6 gluons (n = 8), 2^22 events: weights and d w/d u, d w/d k,
    d w/d ln mu_R (FP32 forward + adjoint amplitude, FP64 boost)."""
    n = 8
    u, hel, order = tess.tess_draws(ctx, n, 1, 0, E)
    proc = tess.process(n, precision=tess.TESS_FP32_CURRENTS)
    f = lambda: tess.tess_gradients(ctx, proc, u, hel, order)
    f()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ts = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        f()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ms = statistics.mean(ts)
    return {"value": E / (ms * 1e-3), "unit": "events/s (weight + all gradients)", "events": E, "ms": ms}


def plan_cap(tess, ctx, proc, n_events):
    """Events per amplitude launch (the chunk capacity) of a call with n_events."""
    info = tess.tess_plan_info(ctx, proc, n_events)
    return -(-n_events // max(info["chunks"], 1))


PIPELINE_SOURCES = ("tess_async.cuh", "tess_bg.cuh", "tess_event.cuh", "tess_f2.cuh", "tess_fused.cuh",
                    "tess_kernels.cuh", "tess_lanes.cuh", "tess_math.cuh", "tess_pair.cuh", "tess_pair_w.cuh",
                    "tess_pipe_launch.cuh", "tess_pipeline.cuh", "tess_wave.cuh", "tess_wavep.cuh")


def kernel_source_hash():
    """sha256 over the sources of the generation pipeline's kernels (the
    pipeline instantiation units and every header they include): a committed
    ncu figure is used only while the kernels it was taken from are
    unchanged."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1002_3446_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name in PIPELINE_SOURCES or (name.startswith("tess_pipe_") and name.endswith(".cu")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def read_traffic(workload, variant, events_per_launch):
    """DRAM bytes per launch of the amplitude kernel from the committed ncu
    capture (profiles/traffic_<workload>.json), scaled to this launch size, or
    None when there is none for this variant or the kernels changed since."""
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != kernel_source_hash():
        return None
    entry = rec.get("by_variant", {}).get(str(variant))
    if not entry:
        return None
    return entry["dram_bytes_per_launch"] * events_per_launch / entry["events_per_launch"]


# ------------------------------------------------------------------ oracle (CPU) arm
def cpu_baseline(wl, budget_s=12.0, events=None, random_pol=False):
    import oracle
    threads = os.cpu_count() or 1
    prec_hel = 0 if wl["hel"] == "sum" else (2 if random_pol else 1)
    kw = dict(hel_mode=prec_hel, pt_min=wl["pt_min"])
    if wl["hist"]:
        obs, nb, lo, hi = wl["hist"]
        kw.update(hist_obs=obs, hist_bins=nb, hist_lo=lo, hist_hi=hi)
    op = oracle.process(wl["n"], **kw)
    if events is None:
        probe = 1 << 12
        t0 = time.perf_counter()
        oracle.generate(op, 1, 0, probe, threads=threads, per_event=False, hist=False)
        rate = probe / max(time.perf_counter() - t0, 1e-6)
        events = int(min(wl["n_events"], max(probe, rate * budget_s)))
    t0 = time.perf_counter()
    oracle.generate(op, 1, 0, events, threads=threads, per_event=True)
    dt = time.perf_counter() - t0
    return {"value": events / dt, "unit": "events/s", "cores": threads, "kind": "oracle",
            "sample": f"events 0..{events - 1} of seed 1 of the same workload ({dt:.1f} s)"}


def workload_metric(wl):
    n = wl["n"]
    return f"events/s (gg->{n - 2}g, {n}-point, {'FP64' if wl['precision'] == 'fp64' else 'FP32 currents'})"


def workload_config(name, wl, N, rp=False, cf=False):
    """The workload description both arms print."""
    n = wl["n"]
    return {"workload": f"{name}: gg->{n - 2} gluons, {N} events per GPU, seed 1, sqrt(S)=14 TeV, "
                        f"pT>{wl['pt_min']:g} |eta|<2.5 dR>0.4, "
                        + ("random real polarisations + ordering sampled" if rp else
                           ("helicities and orderings summed exactly" if wl["hel"] == "sum"
                            else "helicity+ordering sampled"))
                        + (", cut-first (amplitudes only for events passing the cuts)" if cf else ""),
            "events_per_gpu": N, "n_gluons": n}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    n = wl["n"]
    for _ in range(args.warmup):
        cpu_baseline(wl, events=1 << 12)
    vals = []
    for _ in range(args.steps):
        vals.append(cpu_baseline(wl, budget_s=min(8.0, max(1.0, 60.0 / max(1, args.steps)))))
    v = statistics.mean(x["value"] for x in vals)
    line = {
        "impl": "reference",
        "metric": workload_metric(wl),
        "value": v,
        "unit": "events/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": statistics.mean(1e3 * int(x["sample"].split("..")[1].split()[0]) / x["value"] for x in vals),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (counter-based Philox draws, toy gluon PDF)",
        "config": dict(workload_config(args.workload, wl, wl["n_events"]), l2="host cores (the oracle)"),
        "cpu_baseline": {"value": v, "unit": "events/s", "cores": vals[0]["cores"], "kind": "oracle",
                         "sample": vals[0]["sample"]},
        "e2e": {"value": v, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_grad_only(args):
    import torch
    import paper_1002_3446_gb300 as tess
    torch.cuda.set_device(0)
    ctx = tess.tess_init(0)
    for _ in range(max(0, args.warmup - 1)):  # bench_gradients runs one untimed call itself
        bench_gradients(torch, tess, ctx, 1, args.events or (1 << 22))
    r = bench_gradients(torch, tess, ctx, args.steps, args.events or (1 << 22))
    print(json.dumps({"metric": "gg -> 6 gluons gradient events/s", "impl": "tess", **r}), flush=True)
    tess.tess_destroy(ctx)


def main():
    args = parse()
    if args.grad_only:
        run_grad_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_tess(args)


if __name__ == "__main__":
    main()
