"""Pins for the oracle's event weight and accumulation.

* The gg -> gg cross section of the Monte Carlo (exact helicity/ordering sum
  and the sampled estimator) against an independent deterministic
  quadrature of the same cross section built from the textbook closed-form
  matrix element (no Rambo, no recursion, no polarisation vectors).  This
  pins the luminosity Jacobian, flux 1/(2 s), the two-body phase space,
  the identical-particle factor 1/2!, the colour/spin average 1/256, the
  coupling and the GeV^-2 -> pb conversion of the weight (cross-section
  formula at the end of Sec. 3), together with the cut implementation.
* Sec. 4 / Fig. 2: a naive single-precision running sum of many weights
  drifts low; the compensated sum does not.
"""
import math

import numpy as np
import pytest

GEV2_PB = 0.3893793721e9


def _gl(a, b, npts):
    x, w = np.polynomial.legendre.leggauss(npts)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def quadrature_sigma_gg_gg(sqrt_s=14000.0, pt_min=20.0, eta_max=2.5, alphas_mz=0.118, mz=91.19, nf=5):
    S = sqrt_s**2
    tau_min = (2 * pt_min) ** 2 / S
    b0 = (33 - 2 * nf) / (12 * math.pi)

    def f(x):
        return 1.7 * x**-0.2 * (1 - x) ** 5

    def alphas(mu):
        return alphas_mz / (1 + alphas_mz * b0 * np.log(mu**2 / mz**2))

    ct_nodes, ct_w = np.polynomial.legendre.leggauss(200)
    total = 0.0
    # ln(tau) panels, denser near threshold
    edges = np.concatenate([np.linspace(math.log(tau_min), math.log(tau_min) + 2, 41),
                            np.linspace(math.log(tau_min) + 2, 0, 61)[1:]])
    for a, b in zip(edges[:-1], edges[1:]):
        lt, wlt = _gl(a, b, 12)
        for ltau, wl in zip(lt, wlt):
            tau = math.exp(ltau)
            shat = tau * S
            if shat <= (2 * pt_min) ** 2:
                continue
            cpt = math.sqrt(1 - (2 * pt_min) ** 2 / shat)  # pT > pt_min
            ymax = min(eta_max, -ltau / 2)
            # kink where the eta window and the pT window meet
            yk = eta_max - math.atanh(cpt)
            ybreaks = sorted({-ymax, ymax} | ({-yk, yk} if 0 < yk < ymax else set()) | {0.0})
            for ya, yb in zip(ybreaks[:-1], ybreaks[1:]):
                ys, wys = _gl(ya, yb, 16)
                for y, wy in zip(ys, wys):
                    x1, x2 = math.exp(ltau / 2 + y), math.exp(ltau / 2 - y)
                    c = min(cpt, math.tanh(eta_max - abs(y)))
                    if c <= 0:
                        continue
                    ct = 0.5 * c * (ct_nodes + 1)
                    wct = 0.5 * c * ct_w
                    t = -shat * (1 - ct) / 2
                    u = -shat * (1 + ct) / 2
                    s = shat
                    pt = 0.5 * math.sqrt(shat) * np.sqrt(1 - ct**2)
                    g2 = 4 * math.pi * alphas(pt)  # mu_R = H_T / 2 = pT
                    m2 = 1152 * g2**2 * (3 - t * u / s**2 - s * u / t**2 - s * t / u**2)
                    # both signs of cos(theta): factor 2
                    inner = 2 * np.sum(wct * m2) / (16 * math.pi) / 2 / 256
                    total += wl * wy * f(x1) * f(x2) / (2 * shat) * inner
    return total * GEV2_PB


@pytest.fixture(scope="module")
def quad_sigma():
    return quadrature_sigma_gg_gg()


@pytest.mark.parametrize("hel_mode,n_events", [(0, 1 << 16), (1, 1 << 18)])
def test_gg_to_gg_sigma_matches_quadrature(orc, quad_sigma, hel_mode, n_events):
    proc = orc.process(4, hel_mode=hel_mode)
    r = orc.generate(proc, 1, 0, n_events, per_event=False, hist=False)
    sig, err = orc.sigma(r["acc"])
    assert abs(sig - quad_sigma) < 4 * err, (sig, err, quad_sigma)
    assert err / sig < 0.1


def test_weights_zero_iff_failed(orc):
    for n in (4, 6, 9):
        proc = orc.process(n)
        r = orc.generate(proc, 3, 0, 4096, hist=False)
        w, ok = r["weight"], r["pass"].astype(bool)
        assert np.all(w[~ok] == 0)
        # sampled helicities include the vanishing ones, whose |m|^2 is 0 or
        # rounding-small; weights are never negative
        assert np.all(w[ok] >= 0) and np.mean(w[ok] > 0) > 0.5
        assert r["acc"][2] == ok.sum()
        assert math.isclose(r["acc"][0], math.fsum(w), rel_tol=1e-14)


def test_histogram_sums(orc):
    proc = orc.process(5, hist_obs=1, hist_bins=40, hist_lo=200.0, hist_hi=3000.0)
    r = orc.generate(proc, 5, 0, 8192)
    assert math.isclose(r["hist_w"].sum(), r["acc"][0], rel_tol=1e-13)
    ok = r["pass"].astype(bool)
    under = r["weight"][ok & (r["ht"] < 200.0)].sum()
    assert math.isclose(r["hist_w"][0], under, rel_tol=1e-13, abs_tol=1e-300)


def test_generate_is_chunking_invariant(orc):
    proc = orc.process(6)
    a = orc.generate(proc, 8, 100, 3000, threads=1)
    b = orc.generate(proc, 8, 100, 3000, threads=7)
    assert np.array_equal(a["weight"], b["weight"])
    assert math.isclose(a["acc"][0], b["acc"][0], rel_tol=1e-15)
    # an event range split in two gives the same events
    c1 = orc.generate(proc, 8, 100, 1000, threads=2)
    c2 = orc.generate(proc, 8, 1100, 2000, threads=2)
    assert np.array_equal(np.concatenate([c1["weight"], c2["weight"]]), a["weight"])


def test_single_precision_running_sum_drifts(orc):
    """Fig. 2 (first panel): a float32 running sum of ~1e7+ weights loses the
    small increments; the compensated FP64 sum keeps full precision."""
    proc = orc.process(4)
    r = orc.generate(proc, 2, 0, 1 << 14, hist=False)
    w = np.tile(r["weight"], 1 << 10)  # 2^24 weights
    exact = math.fsum(w)
    naive32 = float(np.cumsum(w.astype(np.float32), dtype=np.float32)[-1])
    comp = orc.compensated_sum(w)
    assert abs(naive32 - exact) / exact > 1e-3      # visibly wrong
    assert naive32 < exact                           # underestimates
    assert abs(comp - exact) / exact < 1e-15
