"""Pins for the oracle's Rambo, cuts, observables, alpha_s and PDF.

Rambo is cited (not restated) in Sec. 3 of the paper; the pins are the
properties that define flat massless phase space: momentum conservation,
masslessness, the closed-form volume (checked against the two-body recursion
of phase space by numerical quadrature), the Beta(2, m-2) single-particle
energy spectrum and isotropy.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats


def _rambo_events(orc, m, count, seed=5, sqrt_shat=500.0):
    out = []
    for ev in range(count):
        u = [orc.uniform(seed, ev, j) for j in range(4 * m)]
        out.append(orc.rambo(m, sqrt_shat, u))
    return np.array(out)


@pytest.mark.parametrize("m", [2, 3, 5, 8, 10])
def test_rambo_conservation_and_mass(orc, m):
    rs = 731.0
    p = _rambo_events(orc, m, 200, sqrt_shat=rs)
    tot = p.sum(axis=1)
    # the final boost amplifies rounding by ~gamma^2; for two particles the
    # massless seeds can be nearly collinear (gamma ~ 30 in this sample)
    tol = 1e-12 if m > 2 else 1e-10
    assert np.allclose(tot[:, 0], rs, rtol=tol, atol=0)
    assert np.all(np.abs(tot[:, 1:]) < tol * rs)
    m2 = p[..., 0] ** 2 - (p[..., 1:] ** 2).sum(-1)
    assert np.all(np.abs(m2) < 10 * tol * rs * rs)
    assert np.all(p[..., 0] > 0)


def test_phase_space_volume_closed_forms(orc):
    # two and three massless particles: 1/(8 pi) and s/(256 pi^3)
    for s in [1.0, 37.0, 1.0e6]:
        assert math.isclose(orc.rambo_weight(2, s), 1 / (8 * math.pi), rel_tol=1e-14)
        assert math.isclose(orc.rambo_weight(3, s), s / (256 * math.pi**3), rel_tol=1e-14)


@pytest.mark.parametrize("m", [4, 5, 6, 8, 10])
def test_phase_space_volume_recursion(orc, m):
    # Phi_m(s) = int_0^s ds'/(2 pi) Phi_2(s; 0, s') Phi_{m-1}(s'), with the
    # two-body volume for one massless and one mass^2 = s' system
    # Phi_2 = (1 - s'/s)/(8 pi); integrated numerically from Phi_3.
    # Massless k-body volumes scale as s^(k-2), so each level needs one
    # quadrature: c_k = int_0^1 dt (1 - t)/(8 pi) c_{k-1} t^(k-3) / (2 pi).
    s = 4.0e4
    c = 1 / (256 * math.pi**3)
    for k in range(4, m + 1):
        c, _ = integrate.quad(lambda t: (1 - t) / (8 * math.pi) * c * t ** (k - 3) / (2 * math.pi), 0, 1,
                              epsabs=0, epsrel=1e-13)
    assert math.isclose(orc.rambo_weight(m, s), c * s ** (m - 2), rel_tol=1e-10)


@pytest.mark.parametrize("m", [3, 4, 6])
def test_rambo_energy_spectrum_beta(orc, m):
    # in flat massless m-body phase space x = 2E/sqrt(s) ~ Beta(2, m-2)
    rs = 100.0
    p = _rambo_events(orc, m, 6000, seed=11, sqrt_shat=rs)
    x = 2 * p[:, 0, 0] / rs
    assert stats.kstest(x, stats.beta(2, m - 2).cdf).pvalue > 1e-3
    assert abs(x.mean() - 2 / m) < 5 * stats.beta(2, m - 2).std() / math.sqrt(x.size)


def test_rambo_isotropy(orc):
    p = _rambo_events(orc, 4, 5000, seed=3)
    c = (p[..., 3] / np.linalg.norm(p[..., 1:], axis=-1)).ravel()
    assert abs(c.mean()) < 5 / math.sqrt(3 * c.size)
    assert abs((c**2).mean() - 1 / 3) < 5 * math.sqrt(4 / 45 / c.size)
    phi = np.arctan2(p[..., 2], p[..., 1]).ravel()
    assert stats.kstest((phi + math.pi) / (2 * math.pi), "uniform").pvalue > 1e-3


def _jet(pt, eta, phi):
    # massless momentum from pT, pseudorapidity and azimuth
    return [pt * math.cosh(eta), pt * math.cos(phi), pt * math.sin(phi), pt * math.sinh(eta)]


def test_cuts_hand_built(orc):
    p = np.array([_jet(50.0, 0.3, 0.1), _jet(30.0, -1.2, 2.0), _jet(25.0, 1.9, -2.5)])
    ok, ht, pl, rm = orc.cuts(p, 0.0, 20.0, 2.5, 0.4)
    assert ok
    assert math.isclose(ht, 105.0, rel_tol=1e-12) and math.isclose(pl, 50.0, rel_tol=1e-12)
    dr = []
    etas, phis = [0.3, -1.2, 1.9], [0.1, 2.0, -2.5]
    for i in range(3):
        for j in range(i + 1, 3):
            dphi = abs(phis[i] - phis[j])
            dphi = min(dphi, 2 * math.pi - dphi)
            dr.append(math.hypot(etas[i] - etas[j], dphi))
    assert math.isclose(rm, min(dr), rel_tol=1e-12)
    # each cut fails on its own
    assert not orc.cuts(p, 0.0, 26.0, 2.5, 0.4)[0]             # pT
    assert not orc.cuts(p, 0.7, 20.0, 2.5, 0.4)[0]             # lab |eta| after the boost
    assert orc.cuts(p, -0.5, 20.0, 2.5, 0.4)[0]
    q = np.array([_jet(50.0, 0.3, 0.1), _jet(40.0, 0.5, 0.35)])  # Delta R = sqrt(.04+.0625) = 0.32
    assert not orc.cuts(q, 0.0, 20.0, 2.5, 0.4)[0]
    assert orc.cuts(q, 0.0, 20.0, 2.5, 0.3)[0]
    # azimuth wraps around pi
    r = np.array([_jet(50.0, 0.0, math.pi - 0.05), _jet(40.0, 0.0, -math.pi + 0.05)])
    assert math.isclose(orc.cuts(r, 0.0, 20.0, 2.5, 0.01)[3], 0.1, rel_tol=1e-9)


def test_alphas_one_loop(orc):
    assert math.isclose(orc.alphas(91.19), 0.118, rel_tol=1e-15)
    b0 = 23 / (12 * math.pi)
    for mu in [20.0, 91.19, 500.0, 3000.0]:
        h = 1e-5
        dl = (math.log(orc.alphas(mu * math.exp(h))) - math.log(orc.alphas(mu * math.exp(-h)))) / (2 * h)
        assert math.isclose(dl, -2 * b0 * orc.alphas(mu), rel_tol=1e-7)
    assert orc.alphas(1000.0) < orc.alphas(100.0) < orc.alphas(20.0)


def test_toy_pdf(orc):
    for x in [1e-5, 0.01, 0.3, 0.9]:
        assert math.isclose(orc.xg(x), 1.7 * x**-0.2 * (1 - x) ** 5, rel_tol=1e-14)
    assert orc.xg(1.0) == 0.0


def test_hist_bins(orc):
    lib = orc.lib()
    assert lib.orc_hist_bin(19.999, 50, 20.0, 1020.0) == 0
    assert lib.orc_hist_bin(20.0, 50, 20.0, 1020.0) == 1
    assert lib.orc_hist_bin(39.999, 50, 20.0, 1020.0) == 1
    assert lib.orc_hist_bin(40.0, 50, 20.0, 1020.0) == 2
    assert lib.orc_hist_bin(1019.99, 50, 20.0, 1020.0) == 50
    assert lib.orc_hist_bin(1020.0, 50, 20.0, 1020.0) == 51
    assert lib.orc_hist_bin(float("nan"), 50, 20.0, 1020.0) == 0
