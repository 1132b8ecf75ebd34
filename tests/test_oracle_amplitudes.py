"""Pins for the oracle's polarisation vectors and Berends-Giele amplitudes.

The oracle restates Eq. (BG-recursion) and the W-tensor rewrite of Sec. 3.
Nothing here re-types those equations; the amplitudes are checked against
  * the Parke-Taylor formula for MHV amplitudes (any n),
  * the vanishing of all-equal and one-different helicity amplitudes,
  * gauge invariance (eps_i -> eps_i + c k_i, Sec. 4's gauge check),
  * cyclic, reflection and U(1)-decoupling identities,
  * an explicit sum over individual colour-ordered Feynman diagrams built
    from the vertex tensors (no recursion, no current conservation used),
  * the exact SU(3) colour sum over all colour assignments for n = 4, 5
    (where Sec. 4 states leading colour is exact),
  * the textbook closed form for sum |M|^2(gg -> gg).
Helicity labels: label 0 uses eps_+ of the leg's physical direction; with
that rule every leg (incoming or outgoing) carries all-outgoing helicity
minus its label, so MHV = exactly two legs with the odd label.
"""
import itertools
import math

import numpy as np
import pytest

G = np.diag([1.0, -1.0, -1.0, -1.0])


def mdot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


def phys(k, i):
    return -k[i] if i < 2 else k[i]


def event_point(orc, n, ev, seed=17):
    """All-outgoing momenta of a generated event (pinned Rambo)."""
    return orc.event(orc.process(n), seed, ev)["k"]


def eps_for(orc, k, hel):
    return np.array([orc.polvec(phys(k, i), hel[i]) for i in range(len(k))])


def sij(k, i, j):
    return 2 * mdot(k[i], k[j])


def nonvanishing_hel(rng, n):
    """A random helicity labelling with at least two legs of each label
    (the others vanish identically at tree level)."""
    while True:
        hel = list(rng.integers(0, 2, size=n))
        if 2 <= sum(hel) <= n - 2:
            return hel


# ------------------------------------------------------------ polarisation
def test_polarisation_vectors(orc):
    rng = np.random.default_rng(3)
    for _ in range(20):
        v = rng.normal(size=3)
        p = np.concatenate([[np.linalg.norm(v)], v]) * 37.0
        ep, em = orc.polvec(p, 0), orc.polvec(p, 1)
        for e in (ep, em):
            assert abs(mdot(e, p)) < 1e-13 * p[0]
            assert abs(mdot(e, np.conj(e)) + 1) < 1e-14
            assert abs(mdot(e, e)) < 1e-14
            assert e[0] == 0
        assert np.allclose(np.conj(ep), -em, atol=1e-15)
        # helicity eigenstates: rotating by alpha about p-hat gives exp(-+ i alpha)
        nhat = v / np.linalg.norm(v)
        a = 0.7
        K = np.array([[0, -nhat[2], nhat[1]], [nhat[2], 0, -nhat[0]], [-nhat[1], nhat[0], 0]])
        R = np.eye(3) + math.sin(a) * K + (1 - math.cos(a)) * K @ K
        assert np.allclose(R @ ep[1:], np.exp(-1j * a) * ep[1:], atol=1e-14)
        assert np.allclose(R @ em[1:], np.exp(1j * a) * em[1:], atol=1e-14)
        # completeness: sum_h eps^mu eps*^nu = -g^{mu nu} + (p^mu r^nu + r^mu p^nu)/(p.r), r = (1, -p-hat)
        r = np.concatenate([[1.0], -nhat])
        lhs = np.outer(ep, np.conj(ep)) + np.outer(em, np.conj(em))
        rhs = -G + (np.outer(p, r) + np.outer(r, p)) / mdot(p, r)
        assert np.allclose(lhs, rhs, atol=1e-13)


def test_polarisation_beam_axis(orc):
    for sgn in (1.0, -1.0):
        p = np.array([10.0, 0.0, 0.0, 10.0 * sgn])
        for h in (0, 1):
            e = orc.polvec(p, h)
            assert np.all(np.isfinite(e))
            assert abs(mdot(e, p)) < 1e-14 and abs(mdot(e, np.conj(e)) + 1) < 1e-14


# ------------------------------------------------------------ Parke-Taylor
@pytest.mark.parametrize("n", [4, 5, 6, 7, 8, 10, 12])
def test_parke_taylor_mhv(orc, n):
    rng = np.random.default_rng(n)
    for trial in range(6):
        k = event_point(orc, n, trial)
        order = [0] + list(rng.permutation(np.arange(1, n)))
        i, j = rng.choice(n, size=2, replace=False)
        base = int(rng.integers(2))
        hel = [base] * n
        hel[i] = hel[j] = 1 - base
        m = orc.amp(order, k, eps_for(orc, k, hel))
        a2 = abs(m) ** 2 / 2 ** (n - 2)
        den = 1.0
        for a in range(n):
            den *= abs(sij(k, order[a], order[(a + 1) % n]))
        pt = sij(k, i, j) ** 4 / den
        assert math.isclose(a2, pt, rel_tol=1e-10), (n, trial, a2, pt)


@pytest.mark.parametrize("n", [4, 5, 6, 8, 11])
def test_vanishing_helicity_amplitudes(orc, n):
    rng = np.random.default_rng(100 + n)
    k = event_point(orc, n, 3)
    order = list(range(n))
    ref_hel = [0] * n
    ref_hel[0] = ref_hel[1] = 1
    scale = abs(orc.amp(order, k, eps_for(orc, k, ref_hel)))
    assert scale > 0
    for base in (0, 1):
        assert abs(orc.amp(order, k, eps_for(orc, k, [base] * n))) < 1e-11 * scale
        for odd in range(n):
            hel = [base] * n
            hel[odd] = 1 - base
            assert abs(orc.amp(order, k, eps_for(orc, k, hel))) < 1e-11 * scale


# ------------------------------------------------------------ gauge invariance
@pytest.mark.parametrize("n", [4, 5, 6, 7, 9, 12])
def test_gauge_invariance(orc, n):
    rng = np.random.default_rng(200 + n)
    for trial in range(3):
        k = event_point(orc, n, 10 + trial)
        hel = list(rng.integers(0, 2, size=n))
        order = [0] + list(rng.permutation(np.arange(1, n)))
        eps = eps_for(orc, k, hel)
        m0 = orc.amp(order, k, eps)
        # reference scale: an MHV amplitude at the same point (the sampled
        # helicity may be one of the vanishing ones)
        mhv = [0] * n
        mhv[0] = mhv[1] = 1
        ref = max(abs(m0), abs(orc.amp(order, k, eps_for(orc, k, mhv))))
        for leg in range(n):
            c = complex(*rng.normal(size=2)) / k[leg][0]
            e2 = eps.copy()
            e2[leg] = e2[leg] + c * k[leg]
            m1 = orc.amp(order, k, e2)
            assert abs(m1 - m0) < 1e-10 * ref, (n, leg, m0, m1)


def test_gauge_ratio_is_small(orc):
    # Sec. 4 diagnostic: |K[1].Num[2..n]|^2 / |J[1].Num[2..n]|^2 ~ 0, computed by
    # replacing eps_1 by k_1 in the final contraction
    n = 7
    k = event_point(orc, n, 2)
    hel = [0, 1, 0, 1, 1, 0, 1]
    eps = eps_for(orc, k, hel)
    order = list(range(n))
    m = orc.amp(order, k, eps)
    e2 = eps.copy()
    e2[0] = k[0].astype(complex)
    g = orc.amp(order, k, e2)
    assert abs(g) ** 2 / abs(m) ** 2 < 1e-20


# ------------------------------------------------------------ symmetries
@pytest.mark.parametrize("n", [4, 5, 6, 7, 8, 10])
def test_cyclic_reflection_u1(orc, n):
    rng = np.random.default_rng(300 + n)
    k = event_point(orc, n, 5)
    hel = nonvanishing_hel(rng, n)
    eps = eps_for(orc, k, hel)
    order = [0] + list(rng.permutation(np.arange(1, n)))
    m = orc.amp(order, k, eps)
    scale = abs(m)
    for r in range(1, n):
        rolled = order[r:] + order[:r]
        assert abs(orc.amp(rolled, k, eps) - m) < 1e-10 * scale
    rev = order[::-1]
    assert abs(orc.amp(rev, k, eps) - (-1) ** n * m) < 1e-10 * scale
    # U(1) decoupling: leg order[0] inserted at every position of the others
    others = order[1:]
    tot = 0
    mags = 0
    for pos in range(1, n):
        o = others[:pos] + [order[0]] + others[pos:]
        a = orc.amp(o, k, eps)
        tot += a
        mags += abs(a)
    assert abs(tot) < 1e-10 * mags


@pytest.mark.parametrize("n", [4, 5, 6, 8, 10, 12])
def test_w_tensor_form_equals_recursion(orc, n):
    rng = np.random.default_rng(400 + n)
    for trial in range(3):
        k = event_point(orc, n, 20 + trial)
        hel = nonvanishing_hel(rng, n)
        eps = eps_for(orc, k, hel)
        order = [0] + list(rng.permutation(np.arange(1, n)))
        a0 = orc.amp(order, k, eps, form=0)
        a1 = orc.amp(order, k, eps, form=1)
        assert abs(a1 - a0) < 1e-11 * abs(a0)


# ------------------------------------------------------------ brute force
def _trees(lo, hi):
    """All planar tree diagrams (cubic and quartic vertices) for the
    off-shell current of the contiguous legs lo..hi."""
    if lo == hi:
        return [lo]
    out = []
    for i in range(lo, hi):
        for t1 in _trees(lo, i):
            for t2 in _trees(i + 1, hi):
                out.append((t1, t2))
    for i in range(lo, hi - 1):
        for j in range(i + 1, hi):
            for t1 in _trees(lo, i):
                for t2 in _trees(i + 1, j):
                    for t3 in _trees(j + 1, hi):
                        out.append((t1, t2, t3))
    return out


def _v3(kk, p, q):
    """Colour-ordered three-vertex tensor V^{mu nu rho}(k, p, q), all momenta
    outgoing from the vertex, Tr(T^a T^b) = delta^{ab} normalisation."""
    gi = G
    t = (np.einsum("nr,m->mnr", gi, p - q) + np.einsum("rm,n->mnr", gi, q - kk)
         + np.einsum("mn,r->mnr", gi, kk - p))
    return 1j / math.sqrt(2) * t


def _v4():
    gi = G
    t = (2 * np.einsum("mr,ns->mnrs", gi, gi) - np.einsum("mn,rs->mnrs", gi, gi)
         - np.einsum("ms,nr->mnrs", gi, gi))
    return 1j / 2 * t


def _vertex(children):
    """Amputated vertex contraction V^mu from the children's (J, P)."""
    P = sum(c[1] for c in children)
    low = [G @ c[0] for c in children]
    if len(children) == 2:
        return np.einsum("mnr,n,r->m", _v3(-P, children[0][1], children[1][1]), *low), P
    return np.einsum("mnrs,n,r,s->m", _v4(), *low), P


def _evaluate(tree, legs, k, eps):
    if isinstance(tree, int):
        leg = legs[tree]
        return eps[leg], k[leg]
    ch = [_evaluate(t, legs, k, eps) for t in tree]
    V, P = _vertex(ch)
    return -1j * V / mdot(P, P), P


def brute_force_amp(order, k, eps):
    """sum over individual diagrams of eps_{order[0]} . (root vertex)."""
    n = len(order)
    legs = order[1:]
    tot = 0
    count = 0
    for tree in _trees(0, n - 2):
        ch = [_evaluate(t, legs, k, eps) for t in tree]
        V, _ = _vertex(ch)
        tot += mdot(eps[order[0]], V)
        count += 1
    return tot, count


@pytest.mark.parametrize("n,ndiag", [(4, 3), (5, 10), (6, 38)])
def test_brute_force_feynman_diagrams(orc, n, ndiag):
    rng = np.random.default_rng(500 + n)
    for trial in range(4):
        k = event_point(orc, n, 30 + trial)
        hel = nonvanishing_hel(rng, n)
        eps = eps_for(orc, k, hel)
        order = [0] + list(rng.permutation(np.arange(1, n)))
        bf, count = brute_force_amp(order, k, eps)
        assert count == ndiag
        m = orc.amp(order, k, eps)
        # Dixon-normalised amplitude = i m / 2^{(n-2)/2}
        assert abs(bf - 1j * m / 2 ** ((n - 2) / 2)) < 1e-10 * abs(bf), (n, bf, m)


# ------------------------------------------------------------ colour
def _su3_generators():
    l = np.zeros((8, 3, 3), dtype=complex)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7] = np.diag([1, 1, -2]) / math.sqrt(3)
    T = l / math.sqrt(2)  # Tr(T^a T^b) = delta^{ab}
    assert np.allclose(np.einsum("aij,bji->ab", T, T), np.eye(8))
    return T


@pytest.mark.parametrize("n", [4, 5])
def test_full_colour_sum_equals_leading_colour(orc, n):
    """sum over all 8^n colours of |sum_sigma Tr(T^a1 T^a_sigma2 ...) A(1,sigma)|^2
    = N^{n-2}(N^2-1) sum_sigma |A(1,sigma)|^2 exactly for n = 4, 5."""
    T = _su3_generators()
    letters = "abcdefgh"[:n]
    idx = "ijklmnop"
    spec = ",".join(f"{letters[q]}{idx[q]}{idx[(q + 1) % n]}" for q in range(n)) + "->" + letters
    tr = np.einsum(spec, *([T] * n))
    rng = np.random.default_rng(600 + n)
    for trial in range(3):
        k = event_point(orc, n, 40 + trial)
        hel = nonvanishing_hel(rng, n)
        eps = eps_for(orc, k, hel)
        M = np.zeros(tr.shape, dtype=complex)
        lc = 0.0
        for sigma in itertools.permutations(range(1, n)):
            order = [0] + list(sigma)
            a = orc.amp(order, k, eps) / 2 ** ((n - 2) / 2)
            # Tr(T^{a_order0} T^{a_order1} ...) as a function of (a_1..a_n)
            axes = [order.index(q) for q in range(n)]
            M += a * np.transpose(tr, axes)
            lc += abs(a) ** 2
        full = np.sum(np.abs(M) ** 2)
        assert math.isclose(full, 3 ** (n - 2) * 8 * lc, rel_tol=1e-11)


def test_gg_to_gg_closed_form(orc):
    """sum over colours and helicities of |M|^2 for gg -> gg equals
    1152 g^4 (3 - tu/s^2 - su/t^2 - st/u^2) (e.g. Ellis-Stirling-Webber)."""
    proc = orc.process(4, hel_mode=0)
    for ev in range(20):
        e = orc.event(proc, 9, ev)
        k = e["k"]
        s, t, u = sij(k, 0, 1), sij(k, 0, 2), sij(k, 0, 3)
        closed = 1152 * (3 - t * u / s**2 - s * u / t**2 - s * t / u**2)
        # s + t + u = 0 holds only to rounding; su/t^2 etc. amplify it near
        # the forward direction, hence 1e-10 rather than 1e-13
        assert math.isclose(3**2 * 8 * e["me2"], closed, rel_tol=1e-10)


# ------------------------------------------------------------ sampling
def test_sampled_helicity_and_ordering_cover_uniformly(orc):
    from scipy import stats
    n = 4
    proc = orc.process(n, hel_mode=1)
    hel = np.zeros(2**n)
    perms = {}
    N = 4000
    for ev in range(N):
        e = orc.event(proc, 23, ev)
        hel[e["hel_bits"]] += 1
        assert e["perm"][0] == 0 and sorted(e["perm"]) == list(range(n))
        key = tuple(e["perm"])
        perms[key] = perms.get(key, 0) + 1
    assert stats.chisquare(hel).pvalue > 1e-3
    assert len(perms) == math.factorial(n - 1)
    assert stats.chisquare(list(perms.values())).pvalue > 1e-3


def test_sampled_estimator_expectation_equals_exact_sum(orc):
    # averaging the sampled estimator over every (ordering, helicity) of one
    # phase-space point reproduces the exact sum of hel_mode 0
    n = 5
    e_sum = orc.event(orc.process(n, hel_mode=0), 31, 7)
    k = e_sum["k"]
    acc = 0.0
    cnt = 0
    for sigma in itertools.permutations(range(1, n)):
        for h in range(2**n):
            hel = [(h >> i) & 1 for i in range(n)]
            a = orc.amp([0] + list(sigma), k, eps_for(orc, k, hel))
            acc += 2**n * math.factorial(n - 1) * abs(a) ** 2 / 2 ** (n - 2)
            cnt += 1
    assert math.isclose(acc / cnt, e_sum["me2"], rel_tol=1e-12)
    e_one = orc.event(orc.process(n, hel_mode=1), 31, 7)
    assert np.array_equal(e_one["k"], k)  # same kinematics in both modes
