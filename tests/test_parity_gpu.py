"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Criteria (all reference values come from the oracle or from mpmath on the
oracle's inputs; nothing is derived from the CUDA path):
  FP64 path, per event: relative difference <= 1e-10 on |A|^2 and on the
    weight, OR, for an event the oracle shows to be ill-conditioned, at most
    16x the relative change that moving every Rambo / x uniform by one ulp
    produces in the oracle's own result (that is the size of difference a
    one-ulp libm discrepancy can cause; such events sit near zeros of the
    amplitude and carry tiny weights).  With identical inputs (tess_me2) the
    fallback is 16x the oracle's own rounding error against a 50-digit
    evaluation.  Events needing the fallback are counted and reported.
  FP32-current path: the error is stated per result, not bounded per event
    (an FP32 evaluation of an event near a zero of the amplitude can be off
    by O(1)); the median, 99th percentile and the weight-weighted mean (the
    quantity that enters sigma) of the per-event relative error against the
    FP64 oracle are asserted at about three times their measured values
    (FP32_MEDIAN, FP32_P99, FP32_WEIGHTED below) and printed.  An event
    whose Rambo boost amplifies the FP32 seeds' rounding beyond BOOST_ALONE
    (8 ulp(FP32) x gamma^2, as for the observables) is held to that bound
    alone and left out of the weight-weighted mean.
  FP64 events that pass only through the ill-conditioning fallback are
    bounded in number (at most ILL_RATE of the compared events) and listed
    with the oracle's Sec. 4 gauge ratio |k^.Num|^2/|eps.Num|^2.
  Amplitudes that vanish at tree level (all labels equal or one different)
    are rounding noise: both sides must be below 1e-20 (FP64) / 1e-6 (FP32)
    of the event's MHV scale |A(legs 1, 2 with the odd label)|^2.
  Observables: relative 1e-10 (Rambo's final boost amplifies rounding for
    two nearly collinear seeds); in the FP32 forms, whose Rambo seeds, cuts
    and observables are FP32, 1e-4 or 8 ulp(FP32) x gamma^2 of the event's
    boost if larger (the boost amplifies the seeds' rounding by up to
    ~gamma^2; flags may then differ within that distance of a threshold).  Cross sections and histogram bins:
    relative 1e-10 plus an absolute 1e-12 of the total.
  A pass flag may differ only when a cut quantity lies within 1e-9 of its
    threshold.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_1002_3446_gb300 as tess  # noqa: E402

RTOL64 = 1e-10
RTOL32 = 1e-4
# FP32-current error statistics per n: about three times the largest value
# measured at that n over every amplitude variant, precision form and
# polarisation kind of these tests (seeded samples of 300-1000 events).  The
# median grows with the recursion depth (about 1e-6 per leg); the 99th
# percentile of a sample this small is set by the few ill-conditioned
# events it happens to hold, so it is bounded per n as measured.
FP32_P99 = {4: 4e-4, 5: 1.5e-3, 6: 3e-3, 7: 5e-3, 8: 3.5e-2, 9: 5e-3, 10: 5e-3, 11: 3e-3, 12: 3.5e-3}
FP32_WEIGHTED = {4: 5e-6, 5: 1.5e-5, 6: 2.5e-5, 7: 4e-5, 8: 5e-5, 9: 3e-5, 10: 4e-5, 11: 4e-5, 12: 4e-5}
# FP32 forms: an event whose seed-rounding bound through the Rambo boost,
# 8 u gamma^2 (u = 2^-24), exceeds this is compared alone against that bound
# and left out of the weight-weighted statistic (gamma above about 11)
BOOST_ALONE = 1e-5
# FP64: share of compared events allowed to need the ill-conditioning fallback
# (measured: 0.19 % at n = 6 over 2^21 events, 0.14 % at n = 10 over 2^22)
ILL_RATE = 5e-3


def fp32_median_bound(n):
    return 3e-6 * (n - 3)


def fp32_stats_ok(st, n):
    return st["median"] < fp32_median_bound(n) and st["p99"] < FP32_P99[n] and st["weighted"] < FP32_WEIGHTED[n]


def oracle_gauge_ratio(orc, r):
    """Sec. 4 gauge check on the oracle alone: |k^ . Num|^2 / |eps . Num|^2
    for the contracted leg (the first of the colour order), k^ = k / E."""
    k, order, h = r["k"], list(r["perm"]), r["hel_bits"]
    n = len(order)
    eps = np.array([orc.polvec(phys(k, i), (h >> i) & 1) for i in range(n)])
    den = abs(orc.amp(order, k, eps)) ** 2
    l0 = int(order[0])
    eps[l0] = k[l0] / abs(k[l0][0])
    return abs(orc.amp(order, k, eps)) ** 2 / den


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "gpu tests need a CUDA device"
    c = tess.tess_init(0)
    yield c
    tess.tess_destroy(c)


def orc_proc(orc, p):
    return orc.process(p.n_gluons, hel_mode=p.helicity_mode, sqrt_s=p.sqrt_s, pt_min=p.pt_min, eta_max=p.eta_max,
                       dr_min=p.dr_min, alphas_mz=p.alphas_mz, mz=p.mz, nf=p.nf, mu_r_factor=p.mu_r_factor,
                       hist_obs=p.hist_observable, hist_bins=p.hist_bins, hist_lo=p.hist_lo, hist_hi=p.hist_hi)


def gpu_generate(ctx, proc, seed, first, n_events, calls=1):
    run = tess.Run(ctx, proc, n_events)
    for _ in range(calls):
        run.generate(seed, first)
    torch.cuda.synchronize()
    out = {k: (v.cpu().numpy() if v is not None else None) for k, v in run.t.items()}
    out["acc"] = run.acc.cpu().numpy()
    out["sigma"] = run.result()
    if proc.hist_bins > 0:
        out["hist_w"], out["hist_w2"] = run.histograms()
    return out


def vanishing(hel_bits, n):
    c = bin(int(hel_bits)).count("1")
    return c <= 1 or c >= n - 1


def phys(k, i):
    return -k[i] if i < 2 else k[i]


def mhv_scale(orc, k, order):
    n = len(order)
    hel = [0] * n
    hel[0] = hel[1] = 1
    eps = np.array([orc.polvec(phys(k, i), hel[i]) for i in range(n)])
    return abs(orc.amp(list(order), k, eps)) ** 2 / 2 ** (n - 2)


def near_cut(orc, p, k, y, tol=1e-9):
    """True if a cut quantity of the event is within tol (relative) of its threshold."""
    m = p.n_gluons - 2
    pk = k[2:]
    pt = np.hypot(pk[:, 1], pk[:, 2])
    pa = np.linalg.norm(pk[:, 1:], axis=1)
    eta = 0.5 * np.log((pa + pk[:, 3]) / (pa - pk[:, 3])) + y
    if np.any(np.abs(pt / p.pt_min - 1) < tol) or np.any(np.abs(np.abs(eta) - p.eta_max) < tol * p.eta_max):
        return True
    for i in range(m):
        for j in range(i + 1, m):
            dphi = math.atan2(abs(pk[i, 1] * pk[j, 2] - pk[i, 2] * pk[j, 1]), pk[i, 1] * pk[j, 1] + pk[i, 2] * pk[j, 2])
            dr2 = (eta[i] - eta[j]) ** 2 + dphi**2
            if abs(dr2 / p.dr_min**2 - 1) < tol:
                return True
    return False


def ulp_sensitivity(orc, op, seed, ev):
    return orc.ulp_sensitivity(op, seed, ev)


def rambo_gamma(orc, op, seed, ev):
    """Lorentz factor gamma = Q0/M of Rambo's final boost for event ev (from
    its seed momenta): the boost amplifies the FP32 seeds' relative rounding
    by up to ~gamma^2, which sets the FP32 forms' observable tolerance."""
    u = orc.uniforms(op, seed, ev)
    m = op.n - 2
    Q = np.zeros(4)
    for i in range(m):
        a1, a2, b1, b2 = u[2 + 4 * i: 6 + 4 * i]
        c = 2 * a1 - 1
        s = math.sqrt(max(1 - c * c, 0.0))
        q0 = -math.log(b1 * b2)
        Q += q0 * np.array([1.0, s * math.cos(2 * math.pi * a2), s * math.sin(2 * math.pi * a2), c])
    return Q[0] / math.sqrt(max(Q[0] ** 2 - Q[1] ** 2 - Q[2] ** 2 - Q[3] ** 2, 1e-300))


def compare_events(orc, p, g, seed, first, idx, stats=None, events=None):
    """Per-event comparison of GPU outputs at positions idx with the oracle
    (position i holds event first + i, or events[i] when given)."""
    op = orc_proc(orc, p)
    n = p.n_gluons
    fp32 = p.precision in (tess.TESS_FP32_CURRENTS, tess.TESS_FP32_DS)
    floor = RTOL32 if fp32 else RTOL64  # FP32: events above it are only counted
    vtol = 1e-6 if fp32 else 1e-20
    otol = 1e-4 if fp32 else 1e-10  # FP32 form: FP32 Rambo seeds, cuts and observables
    flips = fallback = boosted = 0
    rel = []
    wdiff = wsum = 0.0
    for i in idx:
        ev = first + int(i) if events is None else int(events[i])
        r = orc.event(op, seed, ev)
        etol = otol
        gtol = 0.0
        if fp32:  # FP32 seeds through the boost: a few ulp times gamma^2
            gtol = 8 * 2.0**-24 * rambo_gamma(orc, op, seed, ev) ** 2
            etol = max(otol, gtol)
        for key in ("ht", "ptlead", "rmin"):
            assert np.isclose(g[key][i], r[key], rtol=etol, atol=0), (key, i, g[key][i], r[key], etol)
        if bool(g["pass"][i]) != r["pass"]:
            assert near_cut(orc, p, r["k"], r["y"], etol), f"pass flag differs away from a cut boundary (event {i})"
            flips += 1
            continue
        if p.helicity_mode == tess.TESS_HEL_SAMPLE and vanishing(r["hel_bits"], n):
            # the sampled estimator is 2^n (n-1)! |A|^2
            sc = mhv_scale(orc, r["k"], r["perm"]) * (2**n * math.factorial(n - 1))
            assert abs(g["me2"][i]) <= vtol * sc and abs(r["me2"]) <= vtol * sc, (i, g["me2"][i], r["me2"], sc)
            continue
        e = abs(g["me2"][i] - r["me2"]) / abs(r["me2"])
        if r["pass"]:
            e = max(e, abs(g["weight"][i] - r["weight"]) / abs(r["weight"]))
            if gtol > BOOST_ALONE:
                # the FP32 seeds' rounding through a large boost bounds this
                # event's accuracy, as it bounds its observables: held to that
                # bound (plus the currents' own FP32 bound) alone, not weighted
                # into the sample's statistic (one such event can carry a fifth
                # of a small sample's weight)
                assert e <= gtol + FP32_P99[n], (i, e, gtol)
                boosted += 1
            else:
                wdiff += abs(g["weight"][i] - r["weight"])
                wsum += r["weight"]
        else:
            assert g["weight"][i] == 0.0
        if e > floor:
            if not fp32:
                s = ulp_sensitivity(orc, op, seed, ev)
                assert e <= 16 * s, f"event {i}: relative difference {e:.3e} above 16 x ulp-sensitivity {s:.3e}"
                print(f"  ill-conditioned event {ev}: rel {e:.2e}, ulp sensitivity {s:.2e}, "
                      f"gauge ratio {oracle_gauge_ratio(orc, r):.2e}")
            fallback += 1
        rel.append(e)
    rel = np.array(rel)
    if not fp32:
        assert fallback <= max(1, ILL_RATE * len(rel)), f"{fallback} of {len(rel)} events needed the fallback"
    if stats is not None:
        stats.update(median=float(np.median(rel)), max=float(rel.max()), p99=float(np.quantile(rel, 0.99)),
                     flips=flips, compared=len(rel), ill_conditioned=fallback, boosted=boosted,
                     weighted=wdiff / wsum if wsum > 0 else 0.0)
    return rel


# ---------------------------------------------------------------- amplitude stage
@pytest.mark.parametrize("n", list(range(4, 13)))
@pytest.mark.parametrize("precision", [tess.TESS_FP64, tess.TESS_FP32_CURRENTS])
def test_me2_matches_oracle(ctx, orc, n, precision):
    from mp_reference import amp_exact
    rng = np.random.default_rng(1000 + n)
    E = 300 + n  # several blocks of 128 and a ragged tail
    op = orc.process(n)
    k = np.zeros((E, n, 4))
    order = np.zeros((E, n), dtype=np.uint8)
    hel = np.zeros(E, dtype=np.uint32)
    ref = np.zeros(E)
    epss = []
    for e in range(E):
        k[e] = orc.event(op, 77, e)["k"]
        order[e] = [0] + list(rng.permutation(np.arange(1, n)))
        while True:
            h = int(rng.integers(0, 2**n))
            if not vanishing(h, n):
                break
        hel[e] = h
        eps = np.array([orc.polvec(phys(k[e], i), (h >> i) & 1) for i in range(n)])
        epss.append(eps)
        ref[e] = abs(orc.amp(list(order[e]), k[e], eps)) ** 2 / 2 ** (n - 2)
    dk = torch.tensor(k, device="cuda")
    do = torch.tensor(order, device="cuda")
    dh = torch.tensor(hel.astype(np.int64), device="cuda").to(torch.int32)
    out = torch.empty(E, dtype=torch.float64, device="cuda")
    tess.tess_me2(ctx, n, precision, dk, do, dh, out)
    got = out.cpu().numpy()
    rel = np.abs(got - ref) / np.abs(ref)
    floor = RTOL64 if precision == tess.TESS_FP64 else RTOL32
    ill = 0
    for e in np.nonzero(rel > floor)[0]:
        ill += 1
        if precision == tess.TESS_FP32_CURRENTS:
            continue  # FP32: statistics below
        exact = abs(amp_exact(list(order[e]), k[e], epss[e])) ** 2 / 2 ** (n - 2)
        own = abs(ref[e] - exact) / exact
        assert abs(got[e] - exact) / exact <= max(floor, 16 * own), (e, got[e], ref[e], exact)
    print(f"me2 n={n} precision={precision}: max rel {rel.max():.2e}, median {np.median(rel):.2e}, "
          f"p99 {np.quantile(rel, 0.99):.2e}, {ill} ill-conditioned events")
    if precision == tess.TESS_FP32_CURRENTS:
        assert np.median(rel) < fp32_median_bound(n) and np.quantile(rel, 0.99) < FP32_P99[n]


# ---------------------------------------------------------------- whole event
def test_gg2g_exact_sum_fp64(ctx, orc):
    p = tess.process(4, precision=tess.TESS_FP64, helicity_mode=tess.TESS_HEL_SUM, hist_bins=50)
    N = 3 * 128 * 7 + 45
    g = gpu_generate(ctx, p, 1, 0, N)
    compare_events(orc, p, g, 1, 0, np.arange(N))
    r = orc.generate(orc_proc(orc, p), 1, 0, N)
    assert np.isclose(g["acc"][0] + g["acc"][4], r["acc"][0], rtol=1e-10)
    assert g["acc"][2] == r["acc"][2] and g["acc"][3] == N
    tot = r["hist_w"].sum()
    assert np.allclose(g["hist_w"], r["hist_w"], rtol=1e-10, atol=1e-12 * tot)
    assert np.allclose(g["hist_w2"], r["hist_w2"], rtol=1e-10, atol=1e-12 * r["hist_w2"].sum())


@pytest.mark.parametrize("n", list(range(4, 13)))
def test_sampled_events_fp64(ctx, orc, n):
    p = tess.process(n, precision=tess.TESS_FP64, pt_min=30.0 if n >= 10 else 20.0, hist_bins=40,
                     hist_observable=tess.TESS_OBS_HT, hist_lo=200.0, hist_hi=3000.0)
    N = 2 * 128 + 29 if n >= 10 else 5 * 128 + 29
    first = (1 << 40) + 3
    g = gpu_generate(ctx, p, 5, first, N)
    st = {}
    compare_events(orc, p, g, 5, first, np.arange(N), st)
    print(f"FP64 n={n}: {st}")
    r = orc.generate(orc_proc(orc, p), 5, first, N)
    assert np.isclose(g["acc"][0] + g["acc"][4], r["acc"][0], rtol=1e-10)
    assert np.allclose(g["hist_w"], r["hist_w"], rtol=1e-10, atol=1e-12 * r["hist_w"].sum())


@pytest.mark.parametrize("n", [4, 6, 8, 10, 12])
@pytest.mark.parametrize("precision", [tess.TESS_FP32_CURRENTS, tess.TESS_FP32_DS])
def test_sampled_events_fp32_currents(ctx, orc, n, precision):
    p = tess.process(n, precision=precision, pt_min=30.0 if n >= 10 else 20.0)
    N = 4 * 128 + 17
    g = gpu_generate(ctx, p, 9, 0, N)
    st = {}
    compare_events(orc, p, g, 9, 0, np.arange(N), st)
    print(f"FP32 currents ({'double-single' if precision == tess.TESS_FP32_DS else 'native FP64'} steps) n={n}: "
          f"per-event relative error median {st['median']:.2e} "
          f"p99 {st['p99']:.2e} max {st['max']:.2e} over {st['compared']} events, "
          f"{st['ill_conditioned']} ill-conditioned, {st['flips']} cut flips, "
          f"weight-weighted {st['weighted']:.2e}")
    assert fp32_stats_ok(st, n), st


@pytest.mark.parametrize("n", [4, 5, 6, 8, 10, 12])
def test_random_polarisation_fp64(ctx, orc, n):
    """Random real polarisations (Sec. 3) against the oracle's mode 2, FP64."""
    p = tess.process(n, precision=tess.TESS_FP64, helicity_mode=tess.TESS_POL_RANDOM,
                     pt_min=30.0 if n >= 10 else 20.0, hist_bins=20, hist_observable=tess.TESS_OBS_PTLEAD,
                     hist_lo=20.0, hist_hi=1020.0)
    N = 2 * 128 + 29 if n >= 10 else 4 * 128 + 29
    first = (1 << 33) + 11
    g = gpu_generate(ctx, p, 4, first, N)
    st = {}
    compare_events(orc, p, g, 4, first, np.arange(N), st)
    print(f"random polarisation FP64 n={n}: {st}")
    r = orc.generate(orc_proc(orc, p), 4, first, N)
    assert np.isclose(g["acc"][0] + g["acc"][4], r["acc"][0], rtol=1e-10)
    assert g["acc"][2] == r["acc"][2]
    assert np.allclose(g["hist_w"], r["hist_w"], rtol=1e-10, atol=1e-12 * r["hist_w"].sum())


@pytest.mark.parametrize("n", [4, 6, 8, 10, 12])
@pytest.mark.parametrize("precision", [tess.TESS_FP32_CURRENTS, tess.TESS_FP32_DS])
def test_random_polarisation_fp32(ctx, orc, n, precision):
    p = tess.process(n, precision=precision, helicity_mode=tess.TESS_POL_RANDOM, pt_min=30.0 if n >= 10 else 20.0)
    N = 4 * 128 + 17
    g = gpu_generate(ctx, p, 8, 5, N)
    st = {}
    compare_events(orc, p, g, 8, 5, np.arange(N), st)
    print(f"random polarisation FP32 precision={precision} n={n}: median {st['median']:.2e} p99 {st['p99']:.2e} "
          f"weighted {st['weighted']:.2e} flips {st['flips']}")
    assert fp32_stats_ok(st, n), st


def test_random_polarisation_sigma_matches_helicity_sampling(ctx):
    """Both estimators are unbiased for the same cross section (n = 6,
    2^22 events each, disjoint from any other test's draws)."""
    res = []
    for mode in (tess.TESS_HEL_SAMPLE, tess.TESS_POL_RANDOM):
        p = tess.process(6, precision=tess.TESS_FP32_DS, helicity_mode=mode)
        run = tess.Run(ctx, p, 1 << 22)
        run.generate(31, 0)
        res.append(run.result())
    (s1, e1), (s2, e2) = res[0][:2], res[1][:2]
    print(f"sigma: sampled helicities {s1:.5e} +- {e1:.1e}, random polarisations {s2:.5e} +- {e2:.1e}")
    assert abs(s1 - s2) < 4 * math.hypot(e1, e2)
    assert res[0][2] == res[1][2]  # the same kinematics pass the same cuts


_LANES = ["LANES8", "LANES16", "LANES32"]
FORMS_BY_N = {
    4: ["REG", "REG_HI", "REG_HI4", "REG_HI_PF", "REG_TMA", "REG_TMA_HI", "PAIR32", "PAIR64", "PAIR_W", "FUSED"],
    6: ["REG", "REG_HI", "REG_HI4", "REG_HI_PF", "REG_TMA", "REG_TMA_HI", "FUSED", "ROWS32", "ROWS64", "PAIR32", "PAIR64",
        "PAIR_W", "WAVE",
        "WAVE2", "WAVE2U", "WAVE2P", "WAVE2PU", "WAVE2L"] + _LANES,
    7: ["WAVE", "WAVE2", "WAVE2U", "WAVE2P", "WAVE2PU", "WAVE2L"] + _LANES,
    8: ["REG", "REG_TMA", "ROWS32", "ROWS64", "PAIR32", "PAIR64", "PAIR_W", "WAVE", "WAVE2", "WAVE2U", "WAVE2P", "WAVE2PU", "WAVE2L"]
    + _LANES,
    9: ["WAVE", "WAVE2", "WAVE2U", "WAVE2P", "WAVE2PU", "WAVE2L"] + _LANES,
    10: ["ROWS32", "ROWS64", "PAIR32", "PAIR64", "PAIR_W", "WAVE", "WAVE2", "WAVE2U", "WAVE2P", "WAVE2PU", "WAVE2L"] + _LANES,
    11: ["WAVE", "WAVE2", "WAVE2U", "WAVE2P", "WAVE2PU", "WAVE2L"] + _LANES,
    12: ["ROWS32", "ROWS64", "PAIR32", "PAIR64", "PAIR_W", "WAVE", "WAVE2", "WAVE2U", "WAVE2P", "WAVE2PU", "WAVE2L"] + _LANES,
}


@pytest.mark.parametrize("n,form", [(n, f) for n, fs in FORMS_BY_N.items() for f in fs])
def test_every_amplitude_variant_against_oracle(ctx, orc, n, form):
    """Each amplitude-kernel variant, forced (serial schedule), on sampled
    events against the oracle with the FP32 criteria; 1000 events span
    several tiles of every variant and end in a ragged one."""
    p = tess.process(n, precision=tess.TESS_FP32_DS, pt_min=30.0 if n >= 10 else 20.0)
    code = getattr(tess, "TESS_K2_" + form)
    tess.tess_select_variant(ctx, p, code, tess.TESS_SCHED_SERIAL)
    try:
        assert tess.tess_plan_info(ctx, p, 1000)["variant"] == code
        N = 1000
        g = gpu_generate(ctx, p, 13, 5, N)
    finally:
        tess.tess_select_variant(ctx, p)
    st = {}
    compare_events(orc, p, g, 13, 5, np.arange(N), st)
    print(f"{form} n={n}: median {st['median']:.2e} p99 {st['p99']:.2e} weighted {st['weighted']:.2e}")
    assert fp32_stats_ok(st, n), st


REAL_FORMS_BY_N = {
    4: ["REAL", "REAL_HI", "REG", "PAIR32"],
    6: ["REAL", "REAL_HI", "REG_HI", "ROWS32", "PAIR64"],
    8: ["REAL", "REAL_HI", "ROWS_REAL", "ROWS64", "PAIR32"],
    9: ["REAL", "ROWS_REAL", "ROWS32", "PAIR32"],
    10: ["ROWS_REAL", "ROWS32", "PAIR64"],
    12: ["ROWS_REAL", "PAIR32"],
}


@pytest.mark.parametrize("n,form", [(n, f) for n, fs in REAL_FORMS_BY_N.items() for f in fs])
def test_random_polarisation_variants_against_oracle(ctx, orc, n, form):
    """Random real polarisations through each amplitude variant that takes
    them: the real-current forms and (imaginary parts zero) the complex
    ones, against the oracle's mode 2 with the FP32 criteria."""
    p = tess.process(n, precision=tess.TESS_FP32_DS, helicity_mode=tess.TESS_POL_RANDOM,
                     pt_min=30.0 if n >= 10 else 20.0)
    code = getattr(tess, "TESS_K2_" + form)
    tess.tess_select_variant(ctx, p, code, tess.TESS_SCHED_SERIAL)
    try:
        assert tess.tess_plan_info(ctx, p, 1000)["variant"] == code
        N = 1000
        g = gpu_generate(ctx, p, 17, 3, N)
    finally:
        tess.tess_select_variant(ctx, p)
    st = {}
    compare_events(orc, p, g, 17, 3, np.arange(N), st)
    print(f"random polarisation {form} n={n}: median {st['median']:.2e} p99 {st['p99']:.2e} "
          f"weighted {st['weighted']:.2e}")
    assert fp32_stats_ok(st, n), st


def test_real_forms_refused_for_helicity_vectors(ctx):
    """The real-current forms need real polarisations: with sampled helicities
    the plan falls back to a complex form, and the two polarisation kinds
    keep separate variant choices."""
    ph = tess.process(6, precision=tess.TESS_FP32_DS)
    pr = tess.process(6, precision=tess.TESS_FP32_DS, helicity_mode=tess.TESS_POL_RANDOM)
    try:
        tess.tess_select_variant(ctx, ph, tess.TESS_K2_REAL, tess.TESS_SCHED_SERIAL)
        assert tess.tess_plan_info(ctx, ph, 10000)["variant"] not in (tess.TESS_K2_REAL, tess.TESS_K2_REAL_HI)
        tess.tess_select_variant(ctx, pr, tess.TESS_K2_REAL_HI, tess.TESS_SCHED_SERIAL)
        assert tess.tess_plan_info(ctx, pr, 10000)["variant"] == tess.TESS_K2_REAL_HI
        tess.tess_select_variant(ctx, ph, tess.TESS_K2_REG, tess.TESS_SCHED_SERIAL)
        assert tess.tess_plan_info(ctx, pr, 10000)["variant"] == tess.TESS_K2_REAL_HI
    finally:
        tess.tess_select_variant(ctx, ph)
        tess.tess_select_variant(ctx, pr)


# ---------------------------------------------------------------- full-size configurations
@pytest.mark.slow
def test_full_gg2g_2e20_fp64(ctx, orc):
    """2^20 events, exact helicity/ordering sum, FP64: every event, sigma and
    the 50-bin leading-jet pT histogram against the oracle run on all cores."""
    p = tess.process(4, precision=tess.TESS_FP64, helicity_mode=tess.TESS_HEL_SUM, hist_bins=50)
    N = 1 << 20
    g = gpu_generate(ctx, p, 1, 0, N)
    r = orc.generate(orc_proc(orc, p), 1, 0, N)
    ok = g["pass"].astype(bool) == r["pass"].astype(bool)
    assert (~ok).sum() <= 5
    rel = np.abs(g["weight"][ok] - r["weight"][ok]) / np.maximum(np.abs(r["weight"][ok]), 1e-300)
    rel[r["weight"][ok] == 0] = 0
    op = orc_proc(orc, p)
    over = np.nonzero(rel > RTOL64)[0]
    assert len(over) < 1e-4 * N
    evs = np.nonzero(ok)[0][over]
    for i, e in zip(over, evs):
        assert rel[i] <= 16 * ulp_sensitivity(orc, op, 1, int(e))
    print(f"gg->gg 2^20: max rel {rel.max():.2e}, {len(over)} ill-conditioned events")
    assert np.isclose(g["sigma"][0], orc.sigma(r["acc"])[0], rtol=1e-10)
    assert np.allclose(g["hist_w"], r["hist_w"], rtol=1e-10, atol=1e-12 * r["hist_w"].sum())


@pytest.mark.slow
@pytest.mark.parametrize("n,N,pt,precision", [(6, 1 << 24, 20.0, tess.TESS_FP32_CURRENTS),
                                              (6, 1 << 24, 20.0, tess.TESS_FP32_DS),
                                              (10, 1 << 26, 30.0, tess.TESS_FP32_CURRENTS),
                                              (10, 1 << 26, 30.0, tess.TESS_FP32_DS)])
def test_full_size_sampled_parity(ctx, orc, n, N, pt, precision):
    """Full-size runs in the benchmark's launch configuration (the amplitude
    variant and chunk schedule chosen by the autotuner on a 2^22-event probe,
    as bench.py does); 1024 sampled events are recomputed one by one by the
    oracle; sigma is checked against the sum of the per-event weights."""
    p = tess.process(n, precision=precision, pt_min=pt, hist_bins=40, hist_observable=tess.TESS_OBS_HT,
                     hist_lo=200.0, hist_hi=3000.0)
    run = tess.Run(ctx, p, N, per_event=("weight", "me2", "pass", "ht", "ptlead", "rmin"))
    acc = torch.zeros(tess.TESS_ACC_LEN, dtype=torch.float64, device="cuda")
    tess.tess_autotune(ctx, p, min(N, 1 << 22), acc, run.workspace)
    print("variant/schedule", tess.tess_plan_info(ctx, p, N))
    run.generate(1, 0)
    torch.cuda.synchronize()
    rng = np.random.default_rng(n)
    idx = np.sort(rng.choice(N, size=1024, replace=False))
    g = {k: v[torch.as_tensor(idx, device="cuda")].cpu().numpy() for k, v in run.t.items()}
    op = orc_proc(orc, p)
    errs = []
    for j, i in enumerate(idx):
        r = orc.event(op, 1, int(i))
        if bool(g["pass"][j]) != r["pass"]:
            assert near_cut(orc, p, r["k"], r["y"], 1e-4)
            continue
        if vanishing(r["hel_bits"], n):
            continue
        errs.append(abs(g["me2"][j] - r["me2"]) / r["me2"])
        assert np.isclose(g["ht"][j], r["ht"], rtol=1e-4)
    errs = np.array(errs)
    print(f"n={n} N={N}: sampled FP32 relative error median {np.median(errs):.2e} "
          f"p99 {np.quantile(errs, 0.99):.2e} max {errs.max():.2e}")
    assert np.median(errs) < fp32_median_bound(n) and np.quantile(errs, 0.99) < FP32_P99[n]
    sig = run.result()
    w = run.t["weight"].double()
    assert np.isclose(sig[0], float(w.sum()) / N, rtol=1e-10)
    assert sig[2] == int(run.t["pass"].sum())
    sw, _ = run.histograms()
    assert np.isclose(sw.sum(), float(w.sum()), rtol=1e-10)


@pytest.mark.slow
@pytest.mark.parametrize("n,N,pt", [(6, 1 << 21, 20.0), (10, 1 << 22, 30.0)])
def test_fp64_multichunk_parity(ctx, orc, n, N, pt):
    """The FP64 sampled pipeline over many chunks (kinematics and amplitude
    kernel pairs, partial rows carried across chunks, the loop-form table in
    local memory), in the launch configuration the benchmark's FP64 leg
    uses: every event's |A|^2, weight and flag against the oracle run over
    all events on the host cores, sigma and the 40-bin H_T histogram against
    the oracle's, sigma against the sum of the per-event weights, and a
    strided 4096-event subset through the full per-event comparison
    (observables, vanishing amplitudes, ill-conditioned events)."""
    import draws_np
    p = tess.process(n, precision=tess.TESS_FP64, pt_min=pt, hist_bins=40, hist_observable=tess.TESS_OBS_HT,
                     hist_lo=200.0, hist_hi=3000.0)
    tess.tess_set_chunk_bytes(ctx, 64 << 20)  # many chunks at a size the oracle covers in seconds
    try:
        info = tess.tess_plan_info(ctx, p, N)
        assert info["chunks"] >= 8, info
        seed = 21
        g = gpu_generate(ctx, p, seed, 0, N)
    finally:
        tess.tess_set_chunk_bytes(ctx, 0)
    op = orc_proc(orc, p)
    r = orc.generate(op, seed, 0, N)
    # sigma and histogram against the oracle over all events
    gs, rs = g["sigma"], orc.sigma(r["acc"])
    assert np.isclose(gs[0], rs[0], rtol=1e-10) and np.isclose(gs[1], rs[1], rtol=1e-8)
    assert gs[3] == N
    tot = r["hist_w"].sum()
    assert np.allclose(g["hist_w"], r["hist_w"], rtol=1e-10, atol=1e-12 * tot)
    assert np.allclose(g["hist_w2"], r["hist_w2"], rtol=1e-10, atol=1e-12 * r["hist_w2"].sum())
    # sigma against the GPU's own per-event weights (accumulation across chunks)
    assert np.isclose(gs[0], orc.compensated_sum(g["weight"]) / N, rtol=1e-12)
    # every event: flags, then |A|^2 and weights of the non-vanishing ones
    flips = np.nonzero(g["pass"].astype(bool) != r["pass"].astype(bool))[0]
    assert len(flips) <= 1e-4 * N
    for i in flips:
        e = orc.event(op, seed, int(i))
        assert near_cut(orc, p, e["k"], e["y"]), f"pass flag of event {i} differs away from a cut"
    van = draws_np.vanishing_mask(n, draws_np.helicity_bits(n, seed, 0, N))
    same = g["pass"].astype(bool) == r["pass"].astype(bool)
    cmp = same & ~van
    rel = np.abs(g["me2"] - r["me2"]) / np.abs(r["me2"])
    passing = cmp & r["pass"].astype(bool)
    relw = np.zeros(N)
    relw[passing] = np.abs(g["weight"][passing] - r["weight"][passing]) / r["weight"][passing]
    rel = np.where(cmp, np.maximum(rel, relw), 0.0)
    assert np.all(g["weight"][same & ~r["pass"].astype(bool)] == 0.0)
    over = np.nonzero(rel > RTOL64)[0]
    print(f"FP64 n={n} N={N} in {info['chunks']} chunks: {cmp.sum()} compared, max rel "
          f"{rel.max():.2e}, {len(over)} above 1e-10, {len(flips)} cut flips")
    assert len(over) <= max(1, ILL_RATE * cmp.sum())
    worst = over[np.argsort(rel[over])[::-1][:32]]
    for i in np.union1d(worst, over[:: max(1, len(over) // 32)]):
        e = orc.event(op, seed, int(i))
        sens = ulp_sensitivity(orc, op, seed, int(i))
        print(f"  ill-conditioned event {i}: rel {rel[i]:.2e}, ulp sensitivity {sens:.2e}, "
              f"gauge ratio {oracle_gauge_ratio(orc, e):.2e}")
        assert rel[i] <= 16 * sens
    # vanishing amplitudes: rounding noise on both sides (a strided sample)
    for i in np.nonzero(van & same)[0][:: max(1, int((van & same).sum()) // 256)]:
        e = orc.event(op, seed, int(i))
        sc = mhv_scale(orc, e["k"], e["perm"]) * (2**n * math.factorial(n - 1))
        assert abs(g["me2"][i]) <= 1e-20 * sc and abs(e["me2"]) <= 1e-20 * sc
    # strided subset through the full per-event comparison
    idx = np.arange(0, N, N // 4096)
    gsub = {k: g[k][idx] for k in ("weight", "me2", "pass", "ht", "ptlead", "rmin")}
    st = {}
    compare_events(orc, p, gsub, seed, 0, np.arange(len(idx)), st, events=idx)
    print(f"  strided subset: {st}")


def test_nonfinite_inputs_stay_in_their_events(ctx, orc):
    """Non-finite caller inputs (host-injected, no device fault): events
    whose momenta hold NaN or infinity give non-finite |A|^2 and gauge
    ratios, and every other event of the call is bit-identical to a clean
    call -- nothing leaks across events, lanes or tiles."""
    n, E = 8, 300
    op = orc.process(n)
    rng = np.random.default_rng(5)
    k = np.array([orc.event(op, 3, e)["k"] for e in range(E)])
    order = np.array([[0] + list(rng.permutation(np.arange(1, n))) for _ in range(E)], dtype=np.uint8)
    hel = np.full(E, 0b11, dtype=np.uint32)
    bad = [0, 131, 299]
    kb = k.copy()
    kb[0, 3, 1] = np.nan
    kb[131, 2, 0] = np.inf  # leg 0 is contracted last: its energy enters no current
    kb[299, 5, 2] = -np.inf
    for prec in (tess.TESS_FP64, tess.TESS_FP32_CURRENTS):
        for fn in (tess.tess_me2, tess.tess_gauge_ratio):
            outs = []
            for kk in (k, kb):
                out = torch.empty(E, dtype=torch.float64, device="cuda")
                fn(ctx, n, prec, torch.tensor(kk, device="cuda"), torch.tensor(order, device="cuda"),
                   torch.tensor(hel.astype(np.int64), device="cuda").to(torch.int32), out)
                outs.append(out.cpu().numpy())
            clean, dirty = outs
            good = np.setdiff1d(np.arange(E), bad)
            assert np.all(np.isfinite(clean))
            assert np.array_equal(clean[good], dirty[good])
            assert not np.any(np.isfinite(dirty[bad]))


@pytest.mark.parametrize("precision", [tess.TESS_FP64, tess.TESS_FP32_DS])
def test_nonfinite_uniforms_in_gradients(ctx, precision):
    """NaN uniforms handed to tess_gradients: every cut comparison with NaN
    is false, so those events fail the cuts (weight 0, zero gradients) and
    the other events keep the clean call's values exactly."""
    n, E = 6, 512
    p = tess.process(n, precision=precision)
    nu = 2 + 4 * (n - 2)
    u, hel, order = tess.tess_draws(ctx, n, 7, 0, E)
    ub = u.clone()
    bad = [3, 200, 511]
    ub[3, 0] = float("nan")
    ub[200, 5] = float("nan")
    ub[511, nu - 1] = float("nan")
    res = []
    for uu in (u, ub):
        res.append(tess.tess_gradients(ctx, p, uu, hel, order))
    good = np.setdiff1d(np.arange(E), bad)
    for key in res[0]:
        a, b = res[0][key].cpu().numpy(), res[1][key].cpu().numpy()
        assert np.array_equal(a[good], b[good]), key
        assert np.all(b[bad] == 0.0), key


def test_result_reports_nonfinite_and_stalls(ctx):
    """tess_result's status from the accumulator row: non-finite weights ->
    TESS_E_NUMERICAL, stalled blocks -> TESS_E_CUDA; the cross section is
    filled in either case."""
    acc = torch.tensor([2.0, 3.0, 1.0, 4.0, 0.0, 0.0, 1.0, 0.0], dtype=torch.float64, device="cuda")
    with pytest.raises(tess.TessError) as e:
        tess.tess_result(ctx, acc)
    assert e.value.code == tess.TESS_E_NUMERICAL
    assert tess.tess_result(ctx, acc, allow_nonfinite=True)[0] == 0.5
    acc[7] = 1.0
    with pytest.raises(tess.TessError) as e:
        tess.tess_result(ctx, acc, allow_nonfinite=True)
    assert e.value.code == tess.TESS_E_CUDA


# ---------------------------------------------------------------- edge cases and API behaviour
def test_split_range_accumulates(ctx, orc):
    p = tess.process(6, precision=tess.TESS_FP64, hist_bins=10, hist_lo=20, hist_hi=220)
    a = gpu_generate(ctx, p, 3, 0, 1000)
    run = tess.Run(ctx, p, 400)
    run.generate(3, 0)
    run2 = tess.Run(ctx, p, 600)
    run2.acc.copy_(run.acc)
    run2.hist.copy_(run.hist)
    run2.generate(3, 400)
    torch.cuda.synchronize()
    assert np.isclose(run2.result()[0], a["sigma"][0], rtol=1e-13)
    assert np.array_equal(run2.t["weight"].cpu().numpy(), a["weight"][400:])
    assert run2.result()[3] == 1000


def test_deterministic(ctx):
    p = tess.process(7, precision=tess.TESS_FP32_CURRENTS, hist_bins=20, hist_lo=20, hist_hi=420)
    r1 = tess.Run(ctx, p, 5000)
    r1.generate(11)
    r2 = tess.Run(ctx, p, 5000)
    r2.generate(11)
    torch.cuda.synchronize()
    assert torch.equal(r1.acc, r2.acc) and torch.equal(r1.hist, r2.hist)
    assert torch.equal(r1.t["weight"], r2.t["weight"])


def test_zero_events_is_noop(ctx):
    p = tess.process(5)
    run = tess.Run(ctx, p, 1)
    tess.tess_generate(ctx, p, 1, 0, 0, run.outputs, run.workspace)
    torch.cuda.synchronize()
    assert float(run.acc.abs().sum()) == 0.0


def test_invalid_arguments_rejected(ctx):
    run = tess.Run(ctx, tess.process(6), 16)
    bad = [tess.process(3), tess.process(13), tess.process(6, helicity_mode=tess.TESS_HEL_SUM),
           tess.process(6, precision=7), tess.process(6, sqrt_s=-1.0), tess.process(6, pt_min=float("nan")),
           tess.process(6, hist_bins=5000), tess.process(12, pt_min=2000.0)]
    for p in bad:
        with pytest.raises(tess.TessError) as e:
            tess.tess_generate(ctx, p, 1, 0, 16, run.outputs, run.workspace)
        assert e.value.code in (tess.TESS_E_INVALID, tess.TESS_E_UNSUPPORTED)
    # histogram requested without a buffer
    with pytest.raises(tess.TessError):
        tess.tess_generate(ctx, tess.process(6, hist_bins=4), 1, 0, 16, run.outputs, run.workspace)
    # workspace too small
    small = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(tess.TessError) as e:
        tess.tess_generate(ctx, tess.process(6), 1, 0, 16, run.outputs, small)
    assert e.value.code == tess.TESS_E_WORKSPACE
    # a host buffer is refused before any kernel touches it
    host = np.zeros(16)
    outs = tess.make_outputs(acc=run.acc)
    outs.weight = host.ctypes.data
    with pytest.raises(tess.TessError) as e:
        tess.tess_generate(ctx, tess.process(6), 1, 0, 16, outs, run.workspace)
    assert e.value.code == tess.TESS_E_INVALID
    torch.cuda.synchronize()


def test_host_copies(ctx):
    p = tess.process(5, precision=tess.TESS_FP64)
    run = tess.Run(ctx, p, 300)
    run.generate(2)
    hw = np.zeros(300)
    hp = np.zeros(300, dtype=np.uint8)
    tess.tess_weights(ctx, run.outputs, 300, hw, hp)
    assert np.array_equal(hw, run.t["weight"].cpu().numpy())
    assert np.array_equal(hp, run.t["pass"].cpu().numpy())
