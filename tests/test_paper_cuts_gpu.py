"""The paper's own second workload and precision diagnostic (Sec. 4): jets
with pT > 60 GeV, |eta| < 2.0, Delta R > 0.4, dynamic scale mu = H_T / 2,
H_T and R_min histograms -- the same kernels on a second set of cuts,
against the oracle -- and the gauge check |k^ . Num|^2 / |eps . Num|^2
(current conservation), whose size is the rounding of the evaluation."""
import math

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


def _orc_proc(orc, p):
    return orc.process(p.n_gluons, hel_mode=p.helicity_mode, sqrt_s=p.sqrt_s, pt_min=p.pt_min, eta_max=p.eta_max,
                       dr_min=p.dr_min, alphas_mz=p.alphas_mz, mz=p.mz, nf=p.nf, mu_r_factor=p.mu_r_factor,
                       hist_obs=p.hist_observable, hist_bins=p.hist_bins, hist_lo=p.hist_lo, hist_hi=p.hist_hi)


@pytest.mark.parametrize("n,obs,lo,hi", [(5, tess.TESS_OBS_HT, 100.0, 1500.0), (6, tess.TESS_OBS_RMIN, 0.4, 3.4),
                                         (6, tess.TESS_OBS_HT, 150.0, 2000.0)])
def test_paper_cuts_histograms_fp64(ctx, orc, n, obs, lo, hi):
    p = tess.process(n, precision=tess.TESS_FP64, pt_min=60.0, eta_max=2.0, dr_min=0.4, hist_bins=30,
                     hist_observable=obs, hist_lo=lo, hist_hi=hi)
    N = 3 * 128 * 5 + 77
    run = tess.Run(ctx, p, N)
    run.generate(21, 1000)
    torch.cuda.synchronize()
    hw, hw2 = run.histograms()
    r = orc.generate(_orc_proc(orc, p), 21, 1000, N)
    acc = run.acc.cpu().numpy()
    assert acc[2] == r["acc"][2] and acc[2] > 0
    assert np.isclose(acc[0] + acc[4], r["acc"][0], rtol=1e-10)
    tot = r["hist_w"].sum()
    assert np.allclose(hw, r["hist_w"], rtol=1e-10, atol=1e-12 * tot)
    assert np.allclose(hw2, r["hist_w2"], rtol=1e-10, atol=1e-12 * r["hist_w2"].sum())


def test_paper_cuts_fp32_sigma(ctx, orc):
    """FP32 currents on the paper's cuts: per-event weights within the FP32
    criteria of the parity tests, through the weight-weighted error."""
    n, N = 6, 4 * 128 + 9
    p = tess.process(n, precision=tess.TESS_FP32_DS, pt_min=60.0, eta_max=2.0, dr_min=0.4)
    run = tess.Run(ctx, p, N)
    run.generate(22, 0)
    torch.cuda.synchronize()
    w = run.t["weight"].cpu().numpy()
    op = _orc_proc(orc, p)
    wo = np.array([orc.event(op, 22, e)["weight"] for e in range(N)])
    both = (w > 0) & (wo > 0)
    assert both.sum() > 5 and ((w > 0) != (wo > 0)).sum() <= 1
    assert np.abs(w[both] - wo[both]).sum() / wo[both].sum() < 1e-4


def _inputs(orc, n, E, seed):
    rng = np.random.default_rng(seed)
    op = orc.process(n)
    k = np.zeros((E, n, 4))
    order = np.zeros((E, n), dtype=np.uint8)
    hel = np.zeros(E, dtype=np.uint32)
    for e in range(E):
        k[e] = orc.event(op, seed, e)["k"]
        order[e] = [0] + list(rng.permutation(np.arange(1, n)))
        while True:
            h = int(rng.integers(0, 2 ** n))
            c = bin(h).count("1")
            if 2 <= c <= n - 2:
                break
        hel[e] = h
    return k, order, hel


@pytest.mark.parametrize("n", [4, 6, 8, 10])
def test_gauge_ratio_profile(ctx, orc, n):
    E = 2048
    k, order, hel = _inputs(orc, n, E, 40 + n)
    dk = torch.tensor(k, device="cuda")
    do = torch.tensor(order, device="cuda")
    dh = torch.tensor(hel.astype(np.int64), device="cuda").to(torch.int32)
    prof = {}
    for prec in (tess.TESS_FP64, tess.TESS_FP32_CURRENTS):
        out = torch.empty(E, dtype=torch.float64, device="cuda")
        tess.tess_gauge_ratio(ctx, n, prec, dk, do, dh, out)
        r = out.cpu().numpy()
        assert np.all(np.isfinite(r)) and np.all(r >= 0)
        prof[prec] = np.quantile(r, [0.5, 0.9, 0.99])
    # the oracle's own ratio on a few events (FP64 rounding noise as well)
    orc_r = []
    for e in range(0, E, 256):
        legs = [((-k[e][i]) if i < 2 else k[e][i]) for i in range(n)]
        eps = np.array([orc.polvec(legs[i], (int(hel[e]) >> i) & 1) for i in range(n)])
        den = abs(orc.amp(list(order[e]), k[e], eps)) ** 2
        l0 = int(order[e][0])
        eps[l0] = k[e][l0] / abs(k[e][l0][0])
        orc_r.append(abs(orc.amp(list(order[e]), k[e], eps)) ** 2 / den)
    print(f"gauge ratio n={n}: FP64 median/p90/p99 {prof[tess.TESS_FP64]}, "
          f"FP32 {prof[tess.TESS_FP32_CURRENTS]}, oracle median {np.median(orc_r):.1e}")
    assert prof[tess.TESS_FP64][0] < 1e-20 and np.median(orc_r) < 1e-20
    assert prof[tess.TESS_FP32_CURRENTS][0] < 1e-6
    assert prof[tess.TESS_FP32_CURRENTS][0] > 10 * prof[tess.TESS_FP64][0]
