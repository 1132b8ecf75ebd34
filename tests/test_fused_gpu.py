"""The warp-specialised one-kernel form (TESS_K2_FUSED): a kinematics
warpgroup hands tiles of 128 events to a register-form amplitude warpgroup
through a two-stage ring in shared memory, one launch per chunk.

Checked through the C ABI: per event against the two-kernel pipeline on the
same events (the kinematics are the same double-float code, so flags and
observables agree exactly; the amplitude is the same register form on the same
FP32 inputs), per event against the FP64 oracle with the FP32 criteria, sigma
against the call's own per-event weights, histograms against a re-binning of
the per-event values, bitwise determinism of the sums, invariance under the
chunk size (several launches per call), and event counts that give the blocks
zero, one, two and many tiles (ring stages reused, ragged last tile).
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


def _host(run):
    torch.cuda.synchronize()
    d = {k: v.cpu().numpy() for k, v in run.t.items() if v is not None}
    d["acc"] = run.acc.cpu().numpy()
    return d


def _generate(ctx, p, n, seed, first, form):
    tess.tess_select_variant(ctx, p, form, tess.TESS_SCHED_SERIAL)
    try:
        assert tess.tess_plan_info(ctx, p, n)["variant"] == form
        run = tess.Run(ctx, p, n)
        run.generate(seed, first)
        return run
    finally:
        tess.tess_select_variant(ctx, p)


def _grid(ctx, p, n):
    tess.tess_select_variant(ctx, p, tess.TESS_K2_FUSED, tess.TESS_SCHED_SERIAL)
    try:
        return tess.tess_plan_info(ctx, p, n)["grid"]
    finally:
        tess.tess_select_variant(ctx, p)


@pytest.mark.parametrize("n", [4, 5, 6])
def test_fused_matches_pipeline(ctx, n):
    p = tess.process(n, precision=tess.TESS_FP32_DS, hist_bins=25, hist_observable=tess.TESS_OBS_HT,
                     hist_lo=50.0, hist_hi=1050.0)
    # about five tiles per block: every block reuses both ring stages, ragged last tile
    N = 5 * 128 * _grid(ctx, p, 1 << 20) + 77
    a = _generate(ctx, p, N, 3, 1000, tess.TESS_K2_FUSED)
    b = _generate(ctx, p, N, 3, 1000, tess.TESS_K2_REG_HI)
    ga, gb = _host(a), _host(b)
    for key in ("pass", "ht", "ptlead", "rmin"):
        assert np.array_equal(ga[key], gb[key]), key
    live = ~draws_np.vanishing_mask(n, draws_np.helicity_bits(n, 3, 1000, N))
    rel = np.abs(ga["me2"][live] - gb["me2"][live]) / gb["me2"][live]
    print(f"n={n}: fused vs pipeline |A|^2 median {np.median(rel):.1e} max {rel.max():.1e}")
    assert np.median(rel) < 2e-6 and np.quantile(rel, 0.99) < 1e-3
    assert np.all(ga["weight"][~ga["pass"].astype(bool)] == 0.0)
    sa, sb = a.result(), b.result()
    assert math.isclose(sa[0], float(np.sum(ga["weight"], dtype=np.float64)) / N, rel_tol=1e-12)
    assert sa[2] == int(ga["pass"].sum()) and sa[3] == N
    assert math.isclose(sa[0], sb[0], rel_tol=1e-5)
    # histogram against a host re-binning of the per-event values
    ok = ga["pass"].astype(bool)
    v, w = ga["ht"][ok], ga["weight"][ok]
    t = (v - p.hist_lo) * (p.hist_bins / (p.hist_hi - p.hist_lo))
    idx = np.where(v < p.hist_lo, 0, np.where(t >= p.hist_bins, p.hist_bins + 1, 1 + np.floor(t).astype(int)))
    expect = np.bincount(idx, weights=w, minlength=p.hist_bins + 2)
    hw, _ = a.histograms()
    assert np.allclose(hw, expect, rtol=1e-12, atol=1e-12 * w.sum())


@pytest.mark.parametrize("n", [4, 6])
def test_fused_against_oracle(ctx, orc, n):
    p = tess.process(n, precision=tess.TESS_FP32_DS)
    N = 3 * 128 * _grid(ctx, p, 1 << 20) + 5
    run = _generate(ctx, p, N, 11, 7, tess.TESS_K2_FUSED)
    g = _host(run)
    idx = np.arange(0, N, max(1, N // 600))
    st = {}
    compare_events(orc, p, g, 11, 7, idx, st)
    print(f"fused n={n}: median {st['median']:.2e} p99 {st['p99']:.2e} weighted {st['weighted']:.2e}")
    assert fp32_stats_ok(st, n), st


@pytest.mark.parametrize("N", [1, 100, 128, 129, 1000])
def test_fused_small_counts(ctx, orc, N):
    """Fewer tiles than blocks: most blocks take no tile and flush zeros.
    Per event against the two-kernel pipeline and, for the observables and
    flags, the oracle (the FP32 error statistics need larger samples: the
    oracle test above)."""
    p = tess.process(6, precision=tess.TESS_FP32_DS)
    run = _generate(ctx, p, N, 19, 0, tess.TESS_K2_FUSED)
    ref = _generate(ctx, p, N, 19, 0, tess.TESS_K2_REG_HI)
    g, r = _host(run), _host(ref)
    for key in ("pass", "ht", "ptlead", "rmin"):
        assert np.array_equal(g[key], r[key]), key
    ok = r["me2"] > 0
    assert np.allclose(g["me2"][ok], r["me2"][ok], rtol=1e-6, atol=0.0)
    assert np.allclose(g["weight"], r["weight"], rtol=1e-6, atol=0.0)
    s = run.result()
    assert s[3] == N and s[2] == int(g["pass"].sum())
    assert math.isclose(s[0], float(np.sum(g["weight"], dtype=np.float64)) / N, rel_tol=1e-12, abs_tol=0.0)
    compare_events(orc, p, g, 19, 0, np.arange(N))


def test_fused_sums_deterministic_and_chunk_invariant(ctx):
    p = tess.process(6, precision=tess.TESS_FP32_DS, hist_bins=10, hist_observable=tess.TESS_OBS_PTLEAD,
                     hist_lo=20.0, hist_hi=220.0)
    N = 1 << 20
    a = _generate(ctx, p, N, 5, 0, tess.TESS_K2_FUSED)
    b = _generate(ctx, p, N, 5, 0, tess.TESS_K2_FUSED)
    torch.cuda.synchronize()
    assert torch.equal(a.acc, b.acc) and torch.equal(a.hist, b.hist)
    assert torch.equal(a.t["weight"], b.t["weight"])
    # 16 MB chunks of per-event data: several launches per call
    tess.tess_set_chunk_bytes(ctx, 16 << 20)
    try:
        tess.tess_select_variant(ctx, p, tess.TESS_K2_FUSED, tess.TESS_SCHED_SERIAL)
        try:
            assert tess.tess_plan_info(ctx, p, N)["chunks"] > 1
        finally:
            tess.tess_select_variant(ctx, p)
        c = _generate(ctx, p, N, 5, 0, tess.TESS_K2_FUSED)
    finally:
        tess.tess_set_chunk_bytes(ctx, 0)
    torch.cuda.synchronize()
    assert torch.equal(a.t["weight"], c.t["weight"])
    sa, sc = a.result(), c.result()
    assert math.isclose(sa[0], sc[0], rel_tol=1e-12) and sa[2] == sc[2]
    ha, _ = a.histograms()
    hc, _ = c.histograms()
    assert np.allclose(ha, hc, rtol=1e-12, atol=0.0)


def test_fused_form_only_where_built(ctx):
    """Where the form is not built (FP32 currents with native FP64 steps,
    random polarisations, cut-first, n > 6) the plan falls back to another
    form."""
    p = tess.process(6, precision=tess.TESS_FP32_DS)
    tess.tess_select_variant(ctx, p, tess.TESS_K2_FUSED, tess.TESS_SCHED_SERIAL)
    try:
        info = tess.tess_plan_info(ctx, p, 1 << 22)
        assert info["variant"] == tess.TESS_K2_FUSED
    finally:
        tess.tess_select_variant(ctx, p)
    for q in (tess.process(6, precision=tess.TESS_FP32_CURRENTS),
              tess.process(6, precision=tess.TESS_FP32_DS, helicity_mode=tess.TESS_POL_RANDOM),
              tess.process(6, precision=tess.TESS_FP32_DS, flags=tess.TESS_FLAG_CUT_FIRST),
              tess.process(8, precision=tess.TESS_FP32_DS)):
        tess.tess_select_variant(ctx, q, tess.TESS_K2_FUSED, tess.TESS_SCHED_SERIAL)
        try:
            assert tess.tess_plan_info(ctx, q, 10000)["variant"] != tess.TESS_K2_FUSED
        finally:
            tess.tess_select_variant(ctx, q)
