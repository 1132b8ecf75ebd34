"""Histograms at the largest bin count (TESS_MAX_BINS): the device's
block-privatised bins and their reduction against a histogram built on the
host from the same run's per-event outputs (weight, H_T, pass), and for the
FP64 form against the oracle's histogram of the same events (Sec. 4's H_T
distribution; bins [lo, hi) plus underflow and overflow)."""
import numpy as np
import pytest
import torch

import paper_1002_3446_gb300 as tess

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "gpu tests need a CUDA device"
    c = tess.tess_init(0)
    yield c
    tess.tess_destroy(c)


def _proc(n, precision):
    return tess.process(n, precision=precision, pt_min=30.0 if n >= 10 else 20.0, hist_bins=tess.TESS_MAX_BINS,
                        hist_observable=tess.TESS_OBS_HT, hist_lo=100.0, hist_hi=2500.0)


def _run(ctx, p, seed, first, N):
    r = tess.Run(ctx, p, N)
    r.generate(seed, first)
    torch.cuda.synchronize()
    hw, hw2 = r.histograms()
    return {k: v.cpu().numpy() for k, v in r.t.items() if v is not None}, np.asarray(hw), np.asarray(hw2), \
        r.acc.cpu().numpy()


def _host_hist(p, ht, w, ok):
    """Bin index 0 (below lo), 1..bins, bins + 1 (at or above hi) of the
    passing events, with the width's reciprocal formed as the library forms it."""
    nb, lo = p.hist_bins, p.hist_lo
    inv = nb / (p.hist_hi - p.hist_lo)
    h, x = ht[ok], w[ok]
    t = (h - lo) * inv
    idx = np.where(h >= lo, np.where(t < nb, 1 + np.floor(np.maximum(t, 0.0)).astype(np.int64), nb + 1), 0)
    return np.bincount(idx, weights=x, minlength=nb + 2), np.bincount(idx, weights=x * x, minlength=nb + 2)


@pytest.mark.parametrize("n,precision,N", [(6, tess.TESS_FP64, 20_000 + 77), (6, tess.TESS_FP32_DS, 300_000 + 77),
                                           (10, tess.TESS_FP32_DS, 100_000 + 77)])
def test_maximum_bins_match_the_per_event_outputs(ctx, n, precision, N):
    p = _proc(n, precision)
    ev, hw, hw2, acc = _run(ctx, p, 11, 1 << 33, N)
    ok = ev["pass"].astype(bool)
    assert ok.sum() > 0
    ref, ref2 = _host_hist(p, ev["ht"], ev["weight"], ok)
    assert hw.shape == (p.hist_bins + 2,)
    # same binning, different summation order
    assert np.allclose(hw, ref, rtol=1e-12, atol=1e-14 * ref.sum())
    assert np.allclose(hw2, ref2, rtol=1e-12, atol=1e-14 * ref2.sum())
    assert np.count_nonzero(hw[1:-1]) > min(p.hist_bins // 8, int(ok.sum()) // 8)
    assert np.isclose(hw.sum(), ev["weight"].sum(), rtol=1e-12)


def test_maximum_bins_fp64_against_oracle(ctx, orc):
    p = _proc(6, tess.TESS_FP64)
    N, first = 3 * 1024 + 5, 12345
    _, hw, hw2, _ = _run(ctx, p, 4, first, N)
    o = orc.generate(orc.process(p.n_gluons, hel_mode=p.helicity_mode, sqrt_s=p.sqrt_s, pt_min=p.pt_min,
                                 eta_max=p.eta_max, dr_min=p.dr_min, alphas_mz=p.alphas_mz, mz=p.mz, nf=p.nf,
                                 mu_r_factor=p.mu_r_factor, hist_obs=p.hist_observable, hist_bins=p.hist_bins,
                                 hist_lo=p.hist_lo, hist_hi=p.hist_hi), 4, first, N)
    assert np.allclose(hw, o["hist_w"], rtol=1e-10, atol=1e-12 * o["hist_w"].sum())
    assert np.allclose(hw2, o["hist_w2"], rtol=1e-10, atol=1e-12 * o["hist_w2"].sum())
