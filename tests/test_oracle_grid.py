"""Pins for the oracle's grid mode (Sec. 3: PDF and alpha_s read from tables
by linear interpolation): node values equal the functions rounded to float,
the interpolation error stays within the linear-interpolation bound
h^2/8 max|f''| (plus float rounding) everywhere, and cross sections with
tables and with the functions agree to that accuracy on the same events."""
import math

import numpy as np


def test_grid_nodes_and_interpolation_bound(orc):
    p = orc.process(6, grid=1)
    lnxmin = math.log((4 * p.pt_min) ** 2 / p.sqrt_s ** 2)
    f = lambda u: orc.xg(math.exp(u * lnxmin))
    for i in (0, 1, 7, 300, 512, 1000, 1023, 1024):
        u = np.float32(i / 1024)
        assert orc.grid_pdf(p, u) == np.float32(f(float(u)))
    # bound: h^2/8 max|f''| over each segment (second differences of a finer
    # sampling), plus a few float roundings of the values
    h = 1 / 1024
    us = np.linspace(0, 1, 16385)
    fs = np.array([f(u) for u in us])
    d2 = np.abs(np.diff(fs, 2)) / (us[1] - us[0]) ** 2
    bound = h * h / 8 * d2.max()
    rng = np.random.default_rng(3)
    worst = 0.0
    for u in rng.uniform(0, 1, 3000).astype(np.float32):
        exact = f(float(u))
        err = abs(orc.grid_pdf(p, u) - exact) - 4 * np.finfo(np.float32).eps * abs(exact)
        worst = max(worst, err / bound)
    assert worst <= 1.0, worst


def test_alphas_grid(orc):
    p = orc.process(8, grid=1)
    m = p.n - 2
    vlo, vhi = 2 * math.log(p.mu_r_factor * m * p.pt_min), 2 * math.log(p.mu_r_factor * p.sqrt_s)
    for i in (0, 100, 512):
        v = vlo + (vhi - vlo) * i / 512
        exact = orc.alphas(math.exp(0.5 * v))
        assert abs(orc.grid_alphas(p, np.float32(v)) - exact) <= 2e-6 * exact
    rng = np.random.default_rng(4)
    for v in rng.uniform(vlo, vhi, 500):
        exact = orc.alphas(math.exp(0.5 * v))
        assert abs(orc.grid_alphas(p, np.float32(v)) - exact) <= 2e-5 * exact  # curvature of 1/log over a step


def test_grid_cross_section_matches_functions(orc):
    n, N = 5, 3000
    ex = orc.process(n)
    gr = orc.process(n, grid=1)
    we = np.array([orc.event(ex, 9, e)["weight"] for e in range(N)])
    wg = np.array([orc.event(gr, 9, e)["weight"] for e in range(N)])
    ok = we > 0
    assert np.array_equal(ok, wg > 0) and ok.sum() > 100
    # linear interpolation of (1 - x)^5 near x -> 1 has a large relative but
    # a negligible absolute error there: compare where the weight matters
    big = we > 1e-6 * we.max()
    rel = np.abs(wg[big] - we[big]) / we[big]
    assert rel.max() < 1e-3 and np.median(rel) < 1e-5 and abs(wg.sum() - we.sum()) < 1e-4 * we.sum()
