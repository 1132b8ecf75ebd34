"""Batched mixed multiplicities (the per-process pipelines recorded one after
another as a single chain of one captured CUDA graph) and the
amplitude-kernel autotuner, through the C ABI.

The batched path runs the same kernels with the same plans as separate
tess_generate calls, so its outputs must be identical to them; replaying the
cached graph accumulates a second time; changing an argument re-captures.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_1002_3446_gb300 as tess  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available()
    c = tess.tess_init(0)
    yield c
    tess.tess_destroy(c)


def _procs():
    return [
        tess.process(4, precision=tess.TESS_FP32_CURRENTS, hist_bins=20, hist_observable=tess.TESS_OBS_PTLEAD),
        tess.process(6, precision=tess.TESS_FP64, hist_bins=10, hist_observable=tess.TESS_OBS_HT, hist_lo=100.0,
                     hist_hi=1100.0),
        tess.process(9, precision=tess.TESS_FP32_CURRENTS),
        tess.process(12, precision=tess.TESS_FP32_CURRENTS, pt_min=30.0),
    ]


def _runs(ctx, procs, counts):
    return [tess.Run(ctx, p, n) for p, n in zip(procs, counts)]


def _host(run):
    torch.cuda.synchronize()
    d = {k: v.cpu().numpy() for k, v in run.t.items() if v is not None}
    d["acc"] = run.acc.cpu().numpy()
    d["hist"] = run.hist.cpu().numpy() if run.hist is not None else None
    return d


def test_batched_equals_separate_calls_and_replays(ctx):
    procs = _procs()
    counts = [70000, 9000, 3001, 700]
    seeds = [1, 2, 3, 4]
    firsts = [0, 10, 1 << 33, 5]
    sep = _runs(ctx, procs, counts)
    for r, s, f in zip(sep, seeds, firsts):
        r.generate(s, f)
    bat = _runs(ctx, procs, counts)
    ws_bytes = tess.tess_workspace_size_batched(ctx, procs, counts)
    ws = torch.empty((ws_bytes + 7) // 8, dtype=torch.float64, device="cuda")
    outs = [r.outputs for r in bat]
    tess.tess_generate_batched(ctx, procs, seeds, firsts, counts, outs, ws)
    for a, b in zip(bat, sep):
        ha, hb = _host(a), _host(b)
        for key in ("weight", "me2", "pass", "ht", "ptlead", "rmin", "acc"):
            assert np.array_equal(ha[key], hb[key]), key
        if ha["hist"] is not None:
            assert np.array_equal(ha["hist"], hb["hist"])
    # replay of the cached graph accumulates again
    tess.tess_generate_batched(ctx, procs, seeds, firsts, counts, outs, ws)
    for a, b, n in zip(bat, sep, counts):
        sa, sb = a.result(), b.result()
        assert sa[3] == 2 * n and np.isclose(sa[0], sb[0], rtol=1e-12)
    # a changed argument re-captures
    seeds2 = [11, 12, 13, 14]
    for r in bat:
        r.reset()
    tess.tess_generate_batched(ctx, procs, seeds2, firsts, counts, outs, ws)
    sep2 = _runs(ctx, procs, counts)
    for r, s, f in zip(sep2, seeds2, firsts):
        r.generate(s, f)
    for a, b in zip(bat, sep2):
        assert np.array_equal(_host(a)["weight"], _host(b)["weight"])


def test_batched_with_fused_form_and_deferred_histogram(ctx):
    """The graph chain with the warp-specialised one-kernel form (n = 6) and the
    deferred-histogram schedule (n = 10 with a histogram, n = 4 FP64 with one)
    selected: bit-identical to separate calls with the same selections, and a
    replay accumulates the same sums again."""
    procs = [tess.process(6, precision=tess.TESS_FP32_DS),
             tess.process(10, precision=tess.TESS_FP32_DS, pt_min=30.0, hist_bins=40,
                          hist_observable=tess.TESS_OBS_HT, hist_lo=200.0, hist_hi=2200.0),
             tess.process(4, precision=tess.TESS_FP64, hist_bins=12, hist_observable=tess.TESS_OBS_PTLEAD)]
    sel = [(tess.TESS_K2_FUSED, tess.TESS_SCHED_SERIAL), (tess.TESS_K2_WAVE2U, tess.TESS_SCHED_SERIAL_HIST),
           (-1, tess.TESS_SCHED_SERIAL_HIST)]
    counts = [200_003, 50_001, 30_007]
    seeds, firsts = [21, 22, 23], [0, 1 << 20, 77]
    try:
        for p, (f, sc) in zip(procs, sel):
            tess.tess_select_variant(ctx, p, f, sc)
            info = tess.tess_plan_info(ctx, p, 1000)
            assert (f < 0 or info["variant"] == f) and info["schedule"] == sc
        sep = _runs(ctx, procs, counts)
        for r, sd, f in zip(sep, seeds, firsts):
            r.generate(sd, f)
        bat = _runs(ctx, procs, counts)
        ws_bytes = tess.tess_workspace_size_batched(ctx, procs, counts)
        ws = torch.empty((ws_bytes + 7) // 8, dtype=torch.float64, device="cuda")
        outs = [r.outputs for r in bat]
        tess.tess_generate_batched(ctx, procs, seeds, firsts, counts, outs, ws)
        for a, b in zip(bat, sep):
            ha, hb = _host(a), _host(b)
            for key in ("weight", "me2", "pass", "ht", "ptlead", "rmin", "acc"):
                assert np.array_equal(ha[key], hb[key]), key
            if ha["hist"] is not None:
                assert np.array_equal(ha["hist"], hb["hist"])
        tess.tess_generate_batched(ctx, procs, seeds, firsts, counts, outs, ws)
        for a, b, n in zip(bat, sep, counts):
            sa, sb = a.result(), b.result()
            assert sa[3] == 2 * n and np.isclose(sa[0], sb[0], rtol=1e-12)
    finally:
        for p in procs:
            tess.tess_select_variant(ctx, p)


def test_batched_rejects_small_workspace(ctx):
    procs = _procs()[:2]
    counts = [1000, 1000]
    bat = _runs(ctx, procs, counts)
    ws = torch.empty(16, dtype=torch.float64, device="cuda")
    with pytest.raises(tess.TessError) as e:
        tess.tess_generate_batched(ctx, procs, [1, 2], [0, 0], counts, [r.outputs for r in bat], ws)
    assert e.value.code == tess.TESS_E_WORKSPACE


@pytest.mark.parametrize("n,prec", [(5, tess.TESS_FP32_CURRENTS), (7, tess.TESS_FP32_CURRENTS),
                                    (8, tess.TESS_FP32_CURRENTS), (10, tess.TESS_FP32_CURRENTS),
                                    (6, tess.TESS_FP64)])
def test_autotune_choice_is_valid_and_consistent(ctx, n, prec):
    proc = tess.process(n, precision=prec, pt_min=30.0 if n >= 10 else 20.0)
    N = 1 << 16
    run = tess.Run(ctx, proc, N)  # workspace sized before tuning
    ref = _host_generate(run)
    acc = torch.zeros(tess.TESS_ACC_LEN, dtype=torch.float64, device="cuda")
    form = tess.tess_autotune(ctx, proc, N, acc, run.workspace)
    valid = {tess.TESS_K2_LOOP} if prec == tess.TESS_FP64 else (
        ({tess.TESS_K2_REG, tess.TESS_K2_REG_TMA} if n <= 8 else set()) | ({tess.TESS_K2_REG_HI, tess.TESS_K2_REG_TMA_HI, tess.TESS_K2_REG_HI_PF} if n <= 7 else set())
        | ({tess.TESS_K2_REG_HI4} if n <= 6 else set())
        | ({tess.TESS_K2_ROWS32, tess.TESS_K2_ROWS64, tess.TESS_K2_WAVE, tess.TESS_K2_WAVE2,
                                                                    tess.TESS_K2_WAVE2U, tess.TESS_K2_WAVE2P,
                                                                    tess.TESS_K2_WAVE2PU, tess.TESS_K2_WAVE2L,
                                                                    tess.TESS_K2_LANES8, tess.TESS_K2_LANES16,
                                                                    tess.TESS_K2_LANES32}
           if n >= 6 else set())
        | {tess.TESS_K2_PAIR32, tess.TESS_K2_PAIR64, tess.TESS_K2_PAIR_W})
    assert form in valid
    run.reset()
    got = _host_generate(run)  # the tuned variant, same workspace
    assert np.array_equal(got["pass"], ref["pass"])
    if prec == tess.TESS_FP64:
        assert np.array_equal(got["weight"], ref["weight"])
    else:
        # variants differ only in the FP32 summation order of the amplitude
        ok = ref["me2"] > 1e-6 * np.median(ref["me2"][ref["me2"] > 0])
        rel = np.abs(got["me2"][ok] - ref["me2"][ok]) / ref["me2"][ok]
        assert np.median(rel) < 1e-5
    print(f"autotune n={n} precision={prec}: variant {form}")


def _host_generate(run):
    run.generate(7, 0)
    return _host(run)


def test_autotune_with_outputs_writes_only_the_per_event_arrays(ctx):
    """tess_autotune_outputs times the variants with the caller's per-event arrays
    written: they hold the probe's events afterwards (the event values do not depend
    on the variant beyond FP32 summation order), acc and hist stay untouched, and the
    choice is a form built for (precision, n)."""
    proc = tess.process(6, precision=tess.TESS_FP32_DS, hist_bins=10, hist_observable=tess.TESS_OBS_HT,
                        hist_lo=100.0, hist_hi=1100.0)
    N = 1 << 17
    run = tess.Run(ctx, proc, N)
    ref = _host_generate(run)
    run.reset()
    for k in ("weight", "me2"):
        run.t[k].fill_(-1.0)
    run.t["pass"].fill_(7)
    form = tess.tess_autotune(ctx, proc, N // 2, None, run.workspace, outputs=run.outputs)
    torch.cuda.synchronize()
    assert form in {tess.TESS_K2_REG, tess.TESS_K2_REG_TMA, tess.TESS_K2_REG_HI, tess.TESS_K2_REG_TMA_HI,
                    tess.TESS_K2_REG_HI_PF, tess.TESS_K2_REG_HI4, tess.TESS_K2_ROWS32, tess.TESS_K2_ROWS64,
                    tess.TESS_K2_WAVE, tess.TESS_K2_WAVE2, tess.TESS_K2_WAVE2U, tess.TESS_K2_WAVE2P,
                    tess.TESS_K2_WAVE2PU, tess.TESS_K2_WAVE2L, tess.TESS_K2_PAIR32, tess.TESS_K2_PAIR64,
                    tess.TESS_K2_PAIR_W, tess.TESS_K2_LANES8, tess.TESS_K2_LANES16, tess.TESS_K2_LANES32,
                    tess.TESS_K2_FUSED}
    assert float(run.acc.abs().sum()) == 0.0 and float(run.hist.abs().sum()) == 0.0
    got = _host(run)
    # the probe draws events [0, N/2) of seed 1
    probe = tess.Run(ctx, proc, N // 2)
    probe.generate(1, 0)
    want = _host(probe)
    h = N // 2
    assert np.array_equal(got["pass"][:h], want["pass"])
    assert np.all(got["pass"][h:] == 7) and np.all(got["weight"][h:] == -1.0)
    ok = want["me2"] > 1e-6 * np.median(want["me2"][want["me2"] > 0])
    rel = np.abs(got["me2"][:h][ok] - want["me2"][ok]) / want["me2"][ok]
    assert np.median(rel) < 1e-5
    assert ref["weight"].shape == got["weight"].shape
    bad = tess.make_outputs(run.t["weight"], None, None, None, None, None, None, None)
    with pytest.raises(tess.TessError) as e:
        tess.tess_autotune(ctx, proc, 1024, None, run.workspace, outputs=bad)
    assert e.value.code == tess.TESS_E_INVALID
