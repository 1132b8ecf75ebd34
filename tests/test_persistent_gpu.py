"""Batched mixed multiplicities in one persistent launch (tess_generate_persistent):
work items (process, 128-event tile) from one atomic counter, partial sums per
tile folded in tile order.

Checked through the C ABI: per event against tess_generate on the same events
(the kinematics are the same double-float form, so flags and observables
agree exactly; the amplitude form differs only in its FP32 summation order),
per event against the FP64 oracle with the FP32 criteria of the parity tests,
sigma against the call's own per-event weights, bitwise determinism of the
sums over repeated calls (whichever block took which tile), histograms
against a re-binning of the per-event values, capture in a CUDA graph, and
the refusals.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import draws_np  # noqa: E402
import paper_1002_3446_gb300 as tess  # noqa: E402
from test_parity_gpu import compare_events, fp32_stats_ok  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available()
    c = tess.tess_init(0)
    yield c
    tess.tess_destroy(c)


def _procs():
    ds = tess.TESS_FP32_DS
    return [
        tess.process(4, precision=ds, hist_bins=20, hist_observable=tess.TESS_OBS_PTLEAD),
        tess.process(6, precision=ds, hist_bins=10, hist_observable=tess.TESS_OBS_HT, hist_lo=100.0, hist_hi=1100.0),
        tess.process(8, precision=ds),
        tess.process(9, precision=ds),
        tess.process(12, precision=ds, pt_min=30.0, hist_bins=40, hist_observable=tess.TESS_OBS_HT, hist_lo=200.0,
                     hist_hi=3000.0),
    ]


COUNTS = [20000, 5003, 1500, 777, 300]  # ragged last tiles
SEEDS = [1, 2, 3, 4, 5]
FIRSTS = [0, 10, 1 << 33, 5, 123]


def _host(run):
    torch.cuda.synchronize()
    d = {k: v.cpu().numpy() for k, v in run.t.items() if v is not None}
    d["acc"] = run.acc.cpu().numpy()
    d["hist"] = run.hist.cpu().numpy() if run.hist is not None else None
    return d


def _persistent(ctx, procs, counts, seeds, firsts, calls=1):
    runs = [tess.Run(ctx, p, n) for p, n in zip(procs, counts)]
    nbytes = tess.tess_workspace_size_persistent(ctx, procs, counts)
    ws = torch.empty((nbytes + 7) // 8, dtype=torch.float64, device="cuda")
    for _ in range(calls):
        tess.tess_generate_persistent(ctx, procs, seeds, firsts, counts, [r.outputs for r in runs], ws)
    return runs, ws


def test_persistent_matches_separate_calls(ctx):
    procs = _procs()
    runs, _ = _persistent(ctx, procs, COUNTS, SEEDS, FIRSTS)
    for p, run, n, seed, first in zip(procs, runs, COUNTS, SEEDS, FIRSTS):
        ref = tess.Run(ctx, p, n)
        ref.generate(seed, first)
        a, b = _host(run), _host(ref)
        for key in ("pass", "ht", "ptlead", "rmin"):
            assert np.array_equal(a[key], b[key]), (p.n_gluons, key)
        # amplitudes: the same inputs, another FP32 summation order (the
        # helicity configurations whose tree amplitude vanishes are FP32
        # rounding noise in both and are left out)
        live = ~draws_np.vanishing_mask(p.n_gluons, draws_np.helicity_bits(p.n_gluons, seed, first, n))
        rel = np.abs(a["me2"][live] - b["me2"][live]) / b["me2"][live]
        print(f"n={p.n_gluons}: persistent vs pipeline |A|^2 median {np.median(rel):.1e} max {rel.max():.1e}")
        assert np.median(rel) < 2e-6 and np.quantile(rel, 0.99) < 1e-3
        assert np.all(a["weight"][~a["pass"].astype(bool)] == 0.0)
        # sigma: the call's sums against its own per-event weights
        sa = run.result()
        assert math.isclose(sa[0], float(np.sum(a["weight"], dtype=np.float64)) / n, rel_tol=1e-12)
        assert sa[2] == int(a["pass"].sum()) and sa[3] == n
        sb = ref.result()
        assert math.isclose(sa[0], sb[0], rel_tol=1e-4)
        if p.hist_bins > 0:
            # histogram bins against a host re-binning of the per-event values
            obs = {tess.TESS_OBS_PTLEAD: "ptlead", tess.TESS_OBS_HT: "ht", tess.TESS_OBS_RMIN: "rmin"}
            v = a[obs[p.hist_observable]][a["pass"].astype(bool)]
            w = a["weight"][a["pass"].astype(bool)]
            t = (v - p.hist_lo) * (p.hist_bins / (p.hist_hi - p.hist_lo))
            idx = np.where(v < p.hist_lo, 0, np.where(t >= p.hist_bins, p.hist_bins + 1, 1 + np.floor(t).astype(int)))
            expect = np.bincount(idx, weights=w, minlength=p.hist_bins + 2)
            hw, _ = run.histograms()
            assert np.allclose(hw, expect, rtol=1e-12, atol=1e-12 * w.sum())


def test_persistent_against_oracle(ctx, orc):
    procs = _procs()
    runs, _ = _persistent(ctx, procs, COUNTS, SEEDS, FIRSTS)
    for p, run, n, seed, first in zip(procs, runs, COUNTS, SEEDS, FIRSTS):
        g = _host(run)
        idx = np.arange(0, n, max(1, n // 200))
        st = {}
        compare_events(orc, p, g, seed, first, idx, st)
        print(f"persistent n={p.n_gluons}: median {st['median']:.2e} p99 {st['p99']:.2e} weighted {st['weighted']:.2e}")
        assert fp32_stats_ok(st, p.n_gluons), st


def test_persistent_sums_are_deterministic(ctx):
    procs = _procs()
    a, _ = _persistent(ctx, procs, COUNTS, SEEDS, FIRSTS)
    b, _ = _persistent(ctx, procs, COUNTS, SEEDS, FIRSTS)
    for ra, rb in zip(a, b):
        torch.cuda.synchronize()
        assert torch.equal(ra.acc, rb.acc)
        if ra.hist is not None:
            assert torch.equal(ra.hist, rb.hist)
        assert torch.equal(ra.t["weight"], rb.t["weight"])
    # a second call accumulates into the same acc: twice the sums
    c, _ = _persistent(ctx, procs, COUNTS, SEEDS, FIRSTS, calls=2)
    for ra, rc in zip(a, c):
        torch.cuda.synchronize()
        assert abs(float(rc.acc[0] + rc.acc[4]) - 2 * float(ra.acc[0] + ra.acc[4])) <= 1e-12 * abs(float(rc.acc[0]))
        assert float(rc.acc[3]) == 2 * float(ra.acc[3])


def test_persistent_in_cuda_graph(ctx):
    procs = _procs()[:3]
    counts, seeds, firsts = COUNTS[:3], SEEDS[:3], FIRSTS[:3]
    ref, _ = _persistent(ctx, procs, counts, seeds, firsts)
    runs = [tess.Run(ctx, p, n) for p, n in zip(procs, counts)]
    nbytes = tess.tess_workspace_size_persistent(ctx, procs, counts)
    ws = torch.empty((nbytes + 7) // 8, dtype=torch.float64, device="cuda")
    outs = [r.outputs for r in runs]
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        tess.tess_generate_persistent(ctx, procs, seeds, firsts, counts, outs, ws, stream=s)
    for r in runs:
        r.reset()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(runs, ref):
        assert torch.equal(a.acc, b.acc)
        assert torch.equal(a.t["weight"], b.t["weight"])


def test_persistent_refusals(ctx):
    run = tess.Run(ctx, tess.process(6, precision=tess.TESS_FP32_DS), 16)
    ws = torch.empty(1 << 16, dtype=torch.float64, device="cuda")
    for bad in (tess.process(6, precision=tess.TESS_FP64), tess.process(6, precision=tess.TESS_FP32_CURRENTS),
                tess.process(5, precision=tess.TESS_FP32_DS, helicity_mode=tess.TESS_HEL_SUM),
                tess.process(6, precision=tess.TESS_FP32_DS, helicity_mode=tess.TESS_POL_RANDOM),
                tess.process(6, precision=tess.TESS_FP32_DS, flags=tess.TESS_FLAG_CUT_FIRST)):
        with pytest.raises(tess.TessError) as e:
            tess.tess_generate_persistent(ctx, [bad], [1], [0], [16], [run.outputs], ws)
        assert e.value.code == tess.TESS_E_UNSUPPORTED
    small = torch.empty(1, dtype=torch.float64, device="cuda")
    p = tess.process(6, precision=tess.TESS_FP32_DS)
    with pytest.raises(tess.TessError) as e:
        tess.tess_generate_persistent(ctx, [p], [1], [0], [16], [run.outputs], small)
    assert e.value.code == tess.TESS_E_WORKSPACE
