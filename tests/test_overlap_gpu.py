"""Chunk schedules: serial or overlapped (kinematics of chunk c+1 on the
caller's stream while the amplitude kernel of chunk c runs on the context's
second stream, two chunk buffers), each with a persistent or a per-tile
amplitude grid, and serial with the histogram deferred to its own kernel per
chunk (the amplitude kernel keeping only the sums).

Every schedule runs the same kernels on the same chunks, so every per-event
output is bit-identical; the accumulated sums differ only in summation order
(the amplitude grid sets it), so they agree to rounding.  Each case spans
several chunks with a ragged last one.
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
    # 16 MB chunks: the cases span several chunks with a ragged last one
    tess.tess_set_chunk_bytes(c, 16 << 20)
    yield c
    tess.tess_destroy(c)


def _host(run):
    torch.cuda.synchronize()
    d = {k: v.cpu().numpy() for k, v in run.t.items() if v is not None}
    d["acc"] = run.acc.cpu().numpy()
    d["hist"] = run.hist.cpu().numpy() if run.hist is not None else None
    return d


CASES = [
    # n, precision, form, events
    (6, tess.TESS_FP32_DS, tess.TESS_K2_REG, 600_001),
    (6, tess.TESS_FP64, tess.TESS_K2_LOOP, 300_017),
    (7, tess.TESS_FP32_CURRENTS, tess.TESS_K2_REG_HI, 500_003),
    (10, tess.TESS_FP32_DS, tess.TESS_K2_ROWS32, 300_001),
    (6, tess.TESS_FP32_DS, tess.TESS_K2_REG_TMA, 600_001),
    (8, tess.TESS_FP32_CURRENTS, tess.TESS_K2_REG_TMA, 400_003),
    (7, tess.TESS_FP32_DS, tess.TESS_K2_REG_TMA_HI, 500_009),
    (10, tess.TESS_FP32_DS, tess.TESS_K2_PAIR32, 300_007),
    (9, tess.TESS_FP32_CURRENTS, tess.TESS_K2_ROWS64, 600_003),
    (6, tess.TESS_FP32_CURRENTS, tess.TESS_K2_PAIR64, 600_011),
    (10, tess.TESS_FP32_DS, tess.TESS_K2_WAVE2U, 300_013),
    (10, tess.TESS_FP32_DS, tess.TESS_K2_WAVE2, 300_019),
    (11, tess.TESS_FP32_DS, tess.TESS_K2_WAVE2P, 200_003),
    (12, tess.TESS_FP32_DS, tess.TESS_K2_LANES8, 200_009),
]


SCHEDS = (tess.TESS_SCHED_SERIAL, tess.TESS_SCHED_OVERLAP, tess.TESS_SCHED_OVERLAP_TILES,
          tess.TESS_SCHED_SERIAL_TILES, tess.TESS_SCHED_SERIAL_HIST)


@pytest.mark.parametrize("n,prec,form,N", CASES)
def test_schedules_match_serial(ctx, n, prec, form, N):
    proc = tess.process(n, precision=prec, pt_min=30.0 if n >= 10 else 20.0, hist_bins=32,
                        hist_observable=tess.TESS_OBS_HT, hist_lo=100.0, hist_hi=2500.0)
    res = {}
    try:
        for sc in SCHEDS:
            tess.tess_select_variant(ctx, proc, form, sc)
            info = tess.tess_plan_info(ctx, proc, N)
            assert info["variant"] == form and info["chunks"] >= 2 and info["schedule"] == sc
            run = tess.Run(ctx, proc, N)
            run.generate(5, 1 << 20)
            first = run.result()
            # a second call into the same outputs must find the first call's buffers retired
            run.generate(6, 1 << 22)
            res[sc] = (_host(run), first, run.result())
            del run
    finally:
        tess.tess_select_variant(ctx, proc)  # back to the default
    b = res[tess.TESS_SCHED_SERIAL]
    for sc in SCHEDS[1:]:
        a = res[sc]
        for key in ("weight", "me2", "pass", "ht", "ptlead", "rmin"):
            assert np.array_equal(a[0][key], b[0][key]), (sc, key)
        for r1, r0 in ((a[1], b[1]), (a[2], b[2])):
            assert r1[2:] == r0[2:]
            assert np.isclose(r1[0], r0[0], rtol=1e-12) and np.isclose(r1[1], r0[1], rtol=1e-10)
        assert np.allclose(a[0]["hist"], b[0]["hist"], rtol=1e-12, atol=1e-14 * np.abs(b[0]["hist"]).sum())


@pytest.mark.parametrize("n", [4, 5, 6, 7, 8])
def test_staged_form_matches_register_form(ctx, n):
    """The staged form reads the same inputs from shared memory instead of
    global memory and evaluates the same amplitude code."""
    proc = tess.process(n, precision=tess.TESS_FP32_DS, hist_bins=16, hist_observable=tess.TESS_OBS_PTLEAD,
                        hist_lo=20.0, hist_hi=500.0)
    N = 300_007
    res = {}
    try:
        forms = (tess.TESS_K2_REG, tess.TESS_K2_REG_TMA) + ((tess.TESS_K2_REG_TMA_HI,) if n <= 7 else ())
        for form in forms:
            tess.tess_select_variant(ctx, proc, form, tess.TESS_SCHED_SERIAL)
            run = tess.Run(ctx, proc, N)
            run.generate(9, 77)
            res[form] = (_host(run), run.result())
    finally:
        tess.tess_select_variant(ctx, proc)
    b = res[tess.TESS_K2_REG]
    for form in forms[1:]:
        a = res[form]
        assert np.array_equal(a[0]["pass"], b[0]["pass"])
        ok = b[0]["me2"] > 0
        rel = np.abs(a[0]["me2"][ok] - b[0]["me2"][ok]) / b[0]["me2"][ok]
        assert np.median(rel) < 1e-6 and np.quantile(rel, 0.99) < 1e-3
        assert a[1][2:] == b[1][2:] and np.isclose(a[1][0], b[1][0], rtol=1e-4)


def test_single_chunk_overlap_runs_serially(ctx):
    proc = tess.process(6, precision=tess.TESS_FP32_DS)
    try:
        tess.tess_select_variant(ctx, proc, -1, tess.TESS_SCHED_OVERLAP)
        assert tess.tess_plan_info(ctx, proc, 1000)["schedule"] == tess.TESS_SCHED_SERIAL
        tess.tess_select_variant(ctx, proc, -1, tess.TESS_SCHED_OVERLAP_TILES)
        assert tess.tess_plan_info(ctx, proc, 1000)["schedule"] == tess.TESS_SCHED_SERIAL_TILES
        run = tess.Run(ctx, proc, 1000)
        run.generate(2, 0)
        assert run.result()[3] == 1000
    finally:
        tess.tess_select_variant(ctx, proc)


def test_overlap_stage_timing_and_batched(ctx):
    procs = [tess.process(6, precision=tess.TESS_FP32_DS), tess.process(8, precision=tess.TESS_FP32_CURRENTS)]
    counts = [500_000, 400_000]
    for p, sc in zip(procs, (tess.TESS_SCHED_OVERLAP, tess.TESS_SCHED_OVERLAP_TILES)):
        tess.tess_select_variant(ctx, p, -1, sc)
    try:
        tess.tess_stage_timing(ctx, True)
        sep = [tess.Run(ctx, p, c) for p, c in zip(procs, counts)]
        for r in sep:
            r.generate(3, 0)
        st = tess.tess_stage_times(ctx)
        tess.tess_stage_timing(ctx, False)
        assert st["kinematics"][1] == st["amplitude"][1] >= 4 and st["amplitude"][0] > 0
        bat = [tess.Run(ctx, p, c) for p, c in zip(procs, counts)]
        ws_bytes = tess.tess_workspace_size_batched(ctx, procs, counts)
        ws = torch.empty((ws_bytes + 7) // 8, dtype=torch.float64, device="cuda")
        tess.tess_generate_batched(ctx, procs, [3, 3], [0, 0], counts, [r.outputs for r in bat], ws)
        for x, y in zip(bat, sep):
            hx, hy = _host(x), _host(y)
            assert np.array_equal(hx["weight"], hy["weight"]) and np.array_equal(hx["acc"], hy["acc"])
    finally:
        for p in procs:
            tess.tess_select_variant(ctx, p)


def test_select_variant_rejects_out_of_range(ctx):
    proc = tess.process(6)
    for form, ov in ((99, 0), (-2, 0), (0, 5), (0, -2)):
        with pytest.raises(tess.TessError) as e:
            tess.tess_select_variant(ctx, proc, form, ov)
        assert e.value.code == tess.TESS_E_INVALID


def test_chunk_size_changes_no_event_and_resizes_the_workspace(ctx):
    """tess_set_chunk_bytes: every event's arithmetic is independent of the chunk
    it lands in, so per-event outputs are bit-identical across chunk sizes and
    the sums agree to rounding (the block partial sums regroup); the workspace
    follows the setting; the batched graph is recaptured after a change; sizes
    below 1 MiB are refused."""
    proc = tess.process(7, precision=tess.TESS_FP32_DS, hist_bins=16, hist_observable=tess.TESS_OBS_HT,
                        hist_lo=100.0, hist_hi=1700.0)
    N = 300_007
    res, ws = {}, {}
    try:
        for mb in (1, 16, 0):
            tess.tess_set_chunk_bytes(ctx, mb << 20)
            info = tess.tess_plan_info(ctx, proc, N)
            ws[mb] = tess.tess_workspace_size(ctx, proc, N)
            run = tess.Run(ctx, proc, N)
            run.generate(9, 77)
            res[mb] = (_host(run), run.result(), info["chunks"])
        assert res[1][2] > res[16][2] > res[0][2] == 1
        assert ws[1] < ws[16] < ws[0]
        for mb in (16, 0):
            for k in ("weight", "me2", "pass", "ht"):
                assert np.array_equal(res[mb][0][k], res[1][0][k]), (mb, k)
            assert res[mb][1][2:] == res[1][1][2:]
            assert np.isclose(res[mb][1][0], res[1][1][0], rtol=1e-12)
            assert np.allclose(res[mb][0]["hist"], res[1][0]["hist"], rtol=1e-12, atol=0)
        # the batched graph follows the setting (recaptured, same events)
        procs, counts = [proc], [N]
        outs = []
        for mb in (1, 0):
            tess.tess_set_chunk_bytes(ctx, mb << 20)
            r = tess.Run(ctx, proc, N)
            nb = tess.tess_workspace_size_batched(ctx, procs, counts)
            w = torch.empty((nb + 7) // 8, dtype=torch.float64, device="cuda")
            tess.tess_generate_batched(ctx, procs, [9], [77], counts, [r.outputs], w)
            outs.append(_host(r))
        assert np.array_equal(outs[0]["weight"], res[1][0]["weight"])
        assert np.array_equal(outs[1]["weight"], res[0][0]["weight"])
        for bad in (1, 4096, (1 << 20) - 1):
            with pytest.raises(tess.TessError) as e:
                tess.tess_set_chunk_bytes(ctx, bad)
            assert e.value.code == tess.TESS_E_INVALID
    finally:
        tess.tess_set_chunk_bytes(ctx, 16 << 20)


def test_deferred_histogram_where_it_applies(ctx):
    """The deferred-histogram schedule against the serial one: with cut-first
    (compacted events) it runs as serial, as it does without a histogram;
    with a histogram and random real polarisations it defers, and the bins
    match a re-binning of the per-event weights."""
    N = 250_007
    for flags, mode, hb in ((tess.TESS_FLAG_CUT_FIRST, tess.TESS_HEL_SAMPLE, 20), (0, tess.TESS_HEL_SAMPLE, 0),
                            (0, tess.TESS_POL_RANDOM, 20)):
        proc = tess.process(8, precision=tess.TESS_FP32_DS, flags=flags, helicity_mode=mode, hist_bins=hb,
                            hist_observable=tess.TESS_OBS_RMIN, hist_lo=0.4, hist_hi=3.4)
        res = {}
        try:
            for sc in (tess.TESS_SCHED_SERIAL, tess.TESS_SCHED_SERIAL_HIST):
                tess.tess_select_variant(ctx, proc, -1, sc)
                run = tess.Run(ctx, proc, N)
                run.generate(3, 11)
                res[sc] = (_host(run), run.result())
        finally:
            tess.tess_select_variant(ctx, proc)
        a, b = res[tess.TESS_SCHED_SERIAL_HIST], res[tess.TESS_SCHED_SERIAL]
        for key in ("weight", "me2", "pass"):
            assert np.array_equal(a[0][key], b[0][key]), key
        assert a[1][2:] == b[1][2:] and np.isclose(a[1][0], b[1][0], rtol=1e-12)
        if hb:
            assert np.allclose(a[0]["hist"], b[0]["hist"], rtol=1e-12, atol=1e-14 * np.abs(b[0]["hist"]).sum())
            ok = a[0]["pass"].astype(bool)
            v, w = a[0]["rmin"][ok], a[0]["weight"][ok]
            t = (v - 0.4) * (hb / 3.0)
            idx = np.where(v < 0.4, 0, np.where(t >= hb, hb + 1, 1 + np.floor(t).astype(int)))
            expect = np.bincount(idx, weights=w, minlength=hb + 2)
            hw, _ = tess.tess_histograms(ctx, proc, torch.from_numpy(a[0]["hist"]).cuda())
            assert np.allclose(hw, expect, rtol=1e-12, atol=1e-12 * w.sum())
