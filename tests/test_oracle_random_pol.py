"""Pins for the oracle's random real polarisation mode (Sec. 3: each
polarisation vector a random unit vector orthogonal to the gluon momentum,
which makes the currents real).

The estimator 2^n |m(eps(phi))|^2 with eps = cos(phi) e1 + sin(phi) e2 must
reproduce the helicity sum; checked here against
  * the defining properties of eps: eps.k = 0, eps.eps = -1, zero time and
    imaginary parts;
  * completeness: the sum of |m|^2 over the 2^n basis choices phi in
    {0, pi/2} equals the sum over the 2^n helicity configurations (a
    unitary change of basis per leg), to rounding;
  * unbiasedness: the mean of 2^n |m|^2 over random angles at a fixed phase
    -space point converges to the helicity sum;
  * the cross section: random polarisations and sampled helicities give the
    same sigma within the Monte Carlo error;
  * the event wiring: the oracle's mode-2 event uses the angle draws at the
    documented positions of the draw layout.
"""
import itertools
import math

import numpy as np


def mdot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


def phys(k, i):
    return -k[i] if i < 2 else k[i]


def test_polvec_real_is_a_transverse_unit_vector(orc):
    rng = np.random.default_rng(5)
    for _ in range(50):
        p3 = rng.normal(size=3) * rng.uniform(1, 500)
        p = np.array([np.linalg.norm(p3), *p3])
        phi = rng.uniform(0, 2 * math.pi)
        e = orc.polvec_real(p, phi)
        assert np.all(e.imag == 0) and e[0] == 0
        assert abs(mdot(e.real, p)) < 1e-12 * p[0]
        assert abs(mdot(e.real, e.real) + 1) < 1e-14
    # beam axis: the fixed basis (e1 = (0, 1, 0, 0) along +z)
    e = orc.polvec_real(np.array([5.0, 0, 0, 5.0]), 0.0)
    assert np.allclose(e.real, [0, 1, 0, 0])


def _sum_hel(orc, n, k, order):
    tot = 0.0
    for hel in itertools.product((0, 1), repeat=n):
        eps = np.array([orc.polvec(phys(k, i), hel[i]) for i in range(n)])
        tot += abs(orc.amp(order, k, eps)) ** 2
    return tot


def test_basis_sum_equals_helicity_sum(orc):
    for n, ev in ((4, 3), (5, 8), (6, 2), (7, 11)):
        k = orc.event(orc.process(n), 23, ev)["k"]
        order = [0] + list(np.random.default_rng(n).permutation(np.arange(1, n)))
        ref = _sum_hel(orc, n, k, order)
        tot = 0.0
        for ang in itertools.product((0.0, 0.5 * math.pi), repeat=n):
            eps = np.array([orc.polvec_real(phys(k, i), ang[i]) for i in range(n)])
            tot += abs(orc.amp(order, k, eps)) ** 2
        assert ref > 0
        assert abs(tot - ref) < 1e-11 * ref, (n, tot, ref)


def test_random_angles_estimate_the_helicity_sum(orc):
    n = 5
    k = orc.event(orc.process(n), 29, 4)["k"]
    order = [0, 2, 4, 1, 3]
    ref = _sum_hel(orc, n, k, order)
    rng = np.random.default_rng(11)
    vals = []
    for _ in range(6000):
        ang = rng.uniform(0, 2 * math.pi, size=n)
        eps = np.array([orc.polvec_real(phys(k, i), ang[i]) for i in range(n)])
        vals.append(2 ** n * abs(orc.amp(order, k, eps)) ** 2)
    vals = np.array(vals)
    err = vals.std() / math.sqrt(len(vals))
    assert abs(vals.mean() - ref) < 4 * err, (vals.mean(), ref, err)
    assert err < 0.05 * ref  # the test has power


def test_sigma_agrees_with_sampled_helicities(orc):
    n, N = 5, 2000000
    res = {}
    for mode in (1, 2):
        r = orc.generate(orc.process(n, hel_mode=mode), 3, 0, N, per_event=False, hist=False)
        acc = r["acc"]
        mean = acc[0] / N
        err = math.sqrt(max(acc[1] / N - mean ** 2, 0) / (N - 1))
        res[mode] = (mean, err)
    (m1, e1), (m2, e2) = res[1], res[2]
    assert abs(m1 - m2) < 4 * math.hypot(e1, e2), res
    assert e2 < 0.08 * m2  # heavy-tailed weights: the error falls slowly


def test_mode2_event_uses_its_angle_draws(orc):
    n = 6
    p1, p2 = orc.process(n, hel_mode=1), orc.process(n, hel_mode=2)
    base = orc.n_uniforms(n, 1)
    assert orc.n_uniforms(n, 2) == base + n
    checked = 0
    for ev in range(40):
        e1, e2 = orc.event(p1, 7, ev), orc.event(p2, 7, ev)
        # x, momenta, cuts and ordering come from the same draws
        assert np.array_equal(e1["k"], e2["k"]) and np.array_equal(e1["perm"], e2["perm"])
        assert e1["pass"] == e2["pass"]
        u = orc.uniforms(p2, 7, ev)
        k, order = e2["k"], e2["perm"]
        eps = np.array([orc.polvec_real(phys(k, i), 2 * math.pi * u[base + i]) for i in range(n)])
        a2 = abs(orc.amp(order, k, eps)) ** 2 / 2 ** (n - 2)
        est = 2 ** n * math.factorial(n - 1) * a2
        if est > 0:
            assert abs(e2["me2"] - est) <= 1e-13 * est
            checked += 1
    assert checked > 30
