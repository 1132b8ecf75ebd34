"""Cut-first generation (TESS_FLAG_CUT_FIRST): the kinematics kernel
compacts the events that pass the cuts and the amplitude kernel evaluates
only those.  Against the plain run of the same events with the same
amplitude variant (itself checked against the oracle): identical weights,
flags and observables event by event, |m|^2 identical for passing events
and 0 for failing ones, and the same sums up to summation order.  Cases span
several chunks with a ragged last one, both FP32 forms, both polarisation
kinds and every schedule."""
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


def _run(ctx, proc, N, seed, first):
    run = tess.Run(ctx, proc, N, per_event=("weight", "me2", "pass", "ht", "ptlead", "rmin"))
    run.generate(seed, first)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in run.t.items() if v is not None}
    out["res"] = run.result()
    out["hist"] = run.hist.cpu().numpy() if run.hist is not None else None
    return out


CASES = [
    # n, precision, helicity mode, form, schedule, events
    (6, tess.TESS_FP32_DS, tess.TESS_HEL_SAMPLE, tess.TESS_K2_REG_HI, tess.TESS_SCHED_OVERLAP, 700_001),
    (6, tess.TESS_FP32_CURRENTS, tess.TESS_HEL_SAMPLE, tess.TESS_K2_REG, tess.TESS_SCHED_SERIAL, 300_007),
    (4, tess.TESS_FP32_DS, tess.TESS_HEL_SAMPLE, tess.TESS_K2_PAIR64, tess.TESS_SCHED_SERIAL_TILES, 500_003),
    (8, tess.TESS_FP32_DS, tess.TESS_POL_RANDOM, tess.TESS_K2_REAL, tess.TESS_SCHED_OVERLAP_TILES, 400_009),
    (10, tess.TESS_FP32_DS, tess.TESS_HEL_SAMPLE, tess.TESS_K2_ROWS64, tess.TESS_SCHED_SERIAL_TILES, 300_011),
    (10, tess.TESS_FP32_DS, tess.TESS_POL_RANDOM, tess.TESS_K2_ROWS_REAL, tess.TESS_SCHED_OVERLAP, 300_013),
    (12, tess.TESS_FP32_DS, tess.TESS_HEL_SAMPLE, tess.TESS_K2_PAIR32, tess.TESS_SCHED_SERIAL, 100_003),
]


@pytest.mark.parametrize("n,prec,mode,form,sched,N", CASES)
def test_cut_first_matches_plain(ctx, n, prec, mode, form, sched, N):
    kw = dict(precision=prec, helicity_mode=mode, pt_min=30.0 if n >= 10 else 20.0, hist_bins=24,
              hist_observable=tess.TESS_OBS_HT, hist_lo=100.0, hist_hi=2500.0)
    plain = tess.process(n, **kw)
    cut = tess.process(n, flags=tess.TESS_FLAG_CUT_FIRST, **kw)
    try:
        for p in (plain, cut):
            tess.tess_select_variant(ctx, p, form, sched)
            info = tess.tess_plan_info(ctx, p, N)
            assert info["variant"] == form and info["schedule"] == sched
        assert tess.tess_plan_info(ctx, cut, N)["chunks"] >= 2 or n == 12
        a = _run(ctx, plain, N, 3, 1 << 20)
        b = _run(ctx, cut, N, 3, 1 << 20)
    finally:
        tess.tess_select_variant(ctx, plain)
        tess.tess_select_variant(ctx, cut)
    ok = a["pass"].astype(bool)
    assert 0 < ok.sum() < N
    diag = {}
    for key in ("weight", "pass", "ht", "ptlead", "rmin", "me2"):
        x, y = a[key], b[key]
        if key == "me2":
            x, y = x[ok], y[ok]
        d = x != y
        rel = np.abs(x[d] - y[d]) / np.maximum(np.abs(x[d]), 1e-300) if d.any() else np.zeros(1)
        diag[key] = (int(d.sum()), float(rel.max()))
    print(f"cut-first n={n} form={form}: differing events (count, max rel) {diag}")
    # the kinematics kernels write out every FP32 rounding of the observables,
    # alpha_s and the weight factor, so the cut-first instantiation gives the
    # same bits as the plain one
    for key in ("weight", "pass", "ht", "ptlead", "rmin", "me2"):
        assert diag[key][0] == 0, (key, diag[key])
    assert np.all(b["me2"][~ok] == 0)
    assert a["res"][2:] == b["res"][2:]  # passing and generated events
    assert np.isclose(a["res"][0], b["res"][0], rtol=1e-12) and np.isclose(a["res"][1], b["res"][1], rtol=1e-10)
    assert np.allclose(a["hist"], b["hist"], rtol=1e-12, atol=1e-14 * np.abs(a["hist"]).sum())


def test_cut_first_variants_and_validation(ctx):
    cut = tess.process(6, precision=tess.TESS_FP32_DS, flags=tess.TESS_FLAG_CUT_FIRST)
    try:
        # the staged (tensor-copy) forms read whole tiles and are not offered
        tess.tess_select_variant(ctx, cut, tess.TESS_K2_REG_TMA, tess.TESS_SCHED_SERIAL)
        assert tess.tess_plan_info(ctx, cut, 100_000)["variant"] != tess.TESS_K2_REG_TMA
    finally:
        tess.tess_select_variant(ctx, cut)
    for bad, code in ((dict(precision=tess.TESS_FP64, flags=tess.TESS_FLAG_CUT_FIRST), tess.TESS_E_UNSUPPORTED),
                      (dict(precision=tess.TESS_FP32_DS, flags=4), tess.TESS_E_INVALID)):
        p = tess.process(6, **bad)
        with pytest.raises(tess.TessError) as e:
            tess.Run(ctx, p, 1000).generate(1, 0)
        assert e.value.code == code
    # autotuning considers only the forms built for it and keeps a separate choice
    plain = tess.process(6, precision=tess.TESS_FP32_DS)
    r = tess.Run(ctx, cut, 1 << 20)
    form = tess.tess_autotune(ctx, cut, 1 << 20, torch.zeros(tess.TESS_ACC_LEN, dtype=torch.float64, device="cuda"),
                              r.workspace)
    assert form not in (tess.TESS_K2_REG_TMA, tess.TESS_K2_REG_TMA_HI)
    tess.tess_select_variant(ctx, plain, tess.TESS_K2_REG_TMA, tess.TESS_SCHED_SERIAL)
    try:
        assert tess.tess_plan_info(ctx, cut, 1 << 20)["variant"] == form
    finally:
        tess.tess_select_variant(ctx, plain)
        tess.tess_select_variant(ctx, cut)
