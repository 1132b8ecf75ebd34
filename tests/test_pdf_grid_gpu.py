"""Grid mode (TESS_FLAG_PDF_GRID, Sec. 3's tabulated PDF and alpha_s with
linear interpolation) against the oracle's grid mode event by event (FP32
criteria of the parity tests), against the function mode (the interpolation
error is small where the weight matters), and combined with the other
flags and modes over several chunks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_1002_3446_gb300 as tess  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available()
    c = tess.tess_init(0)
    # 16 MB chunks: the cases span several chunks
    tess.tess_set_chunk_bytes(c, 16 << 20)
    yield c
    tess.tess_destroy(c)


def _weights(ctx, p, N, seed, first=0):
    run = tess.Run(ctx, p, N)
    run.generate(seed, first)
    torch.cuda.synchronize()
    return run.t["weight"].cpu().numpy(), run.t["pass"].cpu().numpy(), run.result()


@pytest.mark.parametrize("n,prec", [(4, tess.TESS_FP32_DS), (6, tess.TESS_FP32_DS), (6, tess.TESS_FP32_CURRENTS),
                                    (8, tess.TESS_FP32_DS)])
def test_grid_mode_against_oracle(ctx, orc, n, prec):
    N = 3 * 128 + 41
    p = tess.process(n, precision=prec, flags=tess.TESS_FLAG_PDF_GRID)
    w, ok, _ = _weights(ctx, p, N, 12)
    op = orc.process(n, grid=1)
    evs = [orc.event(op, 12, e) for e in range(N)]
    wo = np.array([r["weight"] for r in evs])
    # helicity configurations whose tree amplitude vanishes (all labels equal
    # or one different) are rounding noise on both sides: left out, as in the
    # parity tests
    c = np.array([bin(int(r["hel_bits"])).count("1") for r in evs])
    live = (c >= 2) & (c <= n - 2)
    assert ((w > 0) != (wo > 0)).sum() <= 1
    both = (w > 0) & (wo > 0) & live
    assert both.sum() > 10
    rel = np.abs(w[both] - wo[both]) / wo[both]
    weighted = np.abs(w[both] - wo[both]).sum() / wo[both].sum()
    print(f"grid mode n={n} precision={prec}: median {np.median(rel):.2e} weighted {weighted:.2e}")
    assert np.median(rel) < 1e-5 and weighted < 1e-4


def test_grid_against_functions_and_flags(ctx):
    n, N = 6, 700_001  # several chunks
    base = dict(precision=tess.TESS_FP32_DS, hist_bins=20, hist_observable=tess.TESS_OBS_HT, hist_lo=100.0,
                hist_hi=2100.0)
    wf, okf, rf = _weights(ctx, tess.process(n, **base), N, 5)
    wg, okg, rg = _weights(ctx, tess.process(n, flags=tess.TESS_FLAG_PDF_GRID, **base), N, 5)
    assert np.array_equal(okf, okg)
    big = wf > 1e-6 * wf.max()
    rel = np.abs(wg[big] - wf[big]) / wf[big]
    # (1 - x)^5 interpolated linearly near x -> 1: a larger relative error
    # on the few events there, negligible in sigma
    assert np.median(rel) < 1e-5 and rel.max() < 1e-2
    assert abs(rg[0] - rf[0]) < 1e-4 * rf[0]
    # with cut-first and random polarisations: the same flags per event, and
    # grid + cut-first reproduces grid alone bit for bit
    wc, okc, rc = _weights(ctx, tess.process(n, flags=tess.TESS_FLAG_PDF_GRID | tess.TESS_FLAG_CUT_FIRST, **base),
                           N, 5)
    assert np.array_equal(okc, okg) and np.array_equal(wc, wg)
    wr, okr, _ = _weights(ctx, tess.process(n, helicity_mode=tess.TESS_POL_RANDOM, flags=tess.TESS_FLAG_PDF_GRID,
                                            **base), N, 5)
    assert np.array_equal(okr, okg)


def test_grid_flag_validation(ctx):
    with pytest.raises(tess.TessError) as e:
        tess.Run(ctx, tess.process(6, precision=tess.TESS_FP64, flags=tess.TESS_FLAG_PDF_GRID), 100)
    assert e.value.code == tess.TESS_E_UNSUPPORTED
