"""FP64 gradient oracle: the event weight w(u) of the sampled-mode estimator
restated in plain PyTorch CPU operations (float64 / complex128) so that
torch.autograd supplies its exact derivatives.

TEST INFRASTRUCTURE ONLY (tests import it; the product path never does).
Same method and conventions as tess_oracle.c -- Rambo (Sec. 1, cited),
cuts, one-loop alpha_s, helicity polarisation vectors, Eq. (BG-recursion)
with leg 1 off-shell, leading-colour weight (Sec. 3 cross-section formula)
-- vectorised over events.  Pinned in tests/test_oracle_grad.py against the
C oracle's values and its central finite differences.
"""
from __future__ import annotations

import math

import torch

GEV2_PB = 0.3893793721e9
ETA = torch.tensor([1.0, -1.0, -1.0, -1.0], dtype=torch.float64)


def _mdot(a, b):
    return (a * b * ETA.to(a.dtype)).sum(-1)


def polvec(p, minus):
    """eps_+ = -(e1 + i e2)/sqrt2, eps_- = (e1 - i e2)/sqrt2 of direction p (E,3)."""
    px, py, pz = p[:, 0], p[:, 1], p[:, 2]
    pt2 = px * px + py * py
    beam = pt2 == 0
    # on the beam axis the basis is fixed by convention (phi = 0); keep the
    # masked branch finite so that its (discarded) derivative is not NaN
    pt = torch.sqrt(torch.where(beam, torch.ones_like(pt2), pt2))
    pt = torch.where(beam, torch.zeros_like(pt), pt)
    pa = torch.sqrt(pt2 + pz * pz)
    ct, st = pz / pa, pt / pa
    safe = torch.where(beam, torch.ones_like(pt), pt)
    cf = torch.where(beam, torch.ones_like(pt), px / safe)
    sf = torch.where(beam, torch.zeros_like(pt), py / safe)
    zero = torch.zeros_like(pt)
    e1 = torch.stack([zero, ct * cf, ct * sf, -st], -1)
    e2 = torch.stack([zero, -sf, cf, zero], -1)
    r = 1 / math.sqrt(2.0)
    plus = -(e1 + 1j * e2) * r
    mins = (e1 - 1j * e2) * r
    return torch.where(minus[:, None], mins, plus)


def bg_amplitude(order, k, eps):
    """m = eps_{order[0]} . Num[order[1..]] (paper normalisation), batched.
    order: (E, n) long; k: (E, n, 4) real; eps: (E, n, 4) complex."""
    E, n = order.shape
    L = n - 1
    idx = order[:, 1:]
    lk = torch.gather(k, 1, idx[:, :, None].expand(E, L, 4))
    le = torch.gather(eps, 1, idx[:, :, None].expand(E, L, 4))
    e0 = torch.gather(eps, 1, order[:, :1, None].expand(E, 1, 4))[:, 0]
    J, K = {}, {}
    for a in range(L):
        J[(a, a)] = le[:, a]
        K[(a, a)] = lk[:, a]
    num = None
    for ln in range(2, L + 1):
        for m in range(0, L - ln + 1):
            nn = m + ln - 1
            K[(m, nn)] = K[(m, nn - 1)] + lk[:, nn]
            acc = torch.zeros_like(le[:, 0])
            for i in range(m, nn):
                Ja, Ka, Jb, Kb = J[(m, i)], K[(m, i)], J[(i + 1, nn)], K[(i + 1, nn)]
                acc = acc + (2 * _mdot(Ja, Kb.to(Ja.dtype)))[:, None] * Jb \
                    - (2 * _mdot(Jb, Ka.to(Jb.dtype)))[:, None] * Ja \
                    + _mdot(Ja, Jb)[:, None] * (Ka - Kb).to(Ja.dtype)
            for i in range(m, nn - 1):
                for j in range(i + 1, nn):
                    Ja, Jb, Jc = J[(m, i)], J[(i + 1, j)], J[(j + 1, nn)]
                    acc = acc + (2 * _mdot(Ja, Jc))[:, None] * Jb - _mdot(Ja, Jb)[:, None] * Jc \
                        - _mdot(Jc, Jb)[:, None] * Ja
            if ln < L:
                J[(m, nn)] = acc / _mdot(K[(m, nn)], K[(m, nn)])[:, None]
            else:
                num = acc
    return _mdot(e0, num)


def kinematics(u, n, sqrt_s=14000.0, pt_min=20.0):
    """x1, x2, s_hat and all-outgoing momenta (E, n, 4) from the uniforms."""
    m = n - 2
    S = sqrt_s * sqrt_s
    lnxmin = math.log((m * pt_min) ** 2 / S)
    x1 = torch.exp(u[:, 0] * lnxmin)
    x2 = torch.exp(u[:, 1] * lnxmin)
    shat = x1 * x2 * S
    rs = torch.sqrt(shat)
    ur = u[:, 2:].reshape(-1, m, 4)
    c = 2 * ur[..., 0] - 1
    s = torch.sqrt(1 - c * c)
    phi = 2 * math.pi * ur[..., 1]
    q0 = -torch.log(ur[..., 2] * ur[..., 3])
    q = torch.stack([q0, q0 * s * torch.cos(phi), q0 * s * torch.sin(phi), q0 * c], -1)
    Q = q.sum(1)
    M = torch.sqrt(Q[:, 0] ** 2 - (Q[:, 1:] ** 2).sum(-1))
    b = -Q[:, 1:] / M[:, None]
    gam = Q[:, 0] / M
    a = 1 / (1 + gam)
    x = rs / M
    bq = (b[:, None, :] * q[..., 1:]).sum(-1)
    p0 = x[:, None] * (gam[:, None] * q[..., 0] + bq)
    pv = x[:, None, None] * (q[..., 1:] + b[:, None, :] * (q[..., 0] + a[:, None] * bq)[..., None])
    pout = torch.cat([p0[..., None], pv], -1)
    h = rs / 2
    z = torch.zeros_like(h)
    k1 = torch.stack([-h, z, z, -h], -1)
    k2 = torch.stack([-h, z, z, h], -1)
    k = torch.cat([k1[:, None], k2[:, None], pout], 1)
    return x1, x2, shat, k, lnxmin


def weight(u, hel, order, n, sqrt_s=14000.0, pt_min=20.0, eta_max=2.5, dr_min=0.4, alphas_mz=0.118, mz=91.19,
           nf=5, mu_r_factor=0.5, k_override=None):
    """Per-event weight (pb) of the sampled estimator 2^n (n-1)! |A|^2.
    u: (E, 2+4m) float64; hel: (E,) long; order: (E, n) long.  With
    k_override the momenta are taken as given (x1, x2 still from u)."""
    m = n - 2
    x1, x2, shat, k, lnxmin = kinematics(u, n, sqrt_s, pt_min)
    if k_override is not None:
        k = k_override
    y = 0.5 * torch.log(x1 / x2)
    p = k[:, 2:]
    pt = torch.sqrt(p[..., 1] ** 2 + p[..., 2] ** 2)
    pa = torch.sqrt(p[..., 1] ** 2 + p[..., 2] ** 2 + p[..., 3] ** 2)
    eta = 0.5 * torch.log((pa + p[..., 3]) / (pa - p[..., 3])) + y[:, None]
    ok = ((pt > pt_min) & (eta.abs() < eta_max)).all(1)
    for i in range(m):
        for j in range(i + 1, m):
            dphi = torch.atan2((p[:, i, 1] * p[:, j, 2] - p[:, i, 2] * p[:, j, 1]).abs(),
                               p[:, i, 1] * p[:, j, 1] + p[:, i, 2] * p[:, j, 2])
            ok = ok & ((eta[:, i] - eta[:, j]) ** 2 + dphi ** 2 > dr_min ** 2)
    ht = pt.sum(1)
    b0 = (33 - 2 * nf) / (12 * math.pi)
    mu = mu_r_factor * ht
    alphas = alphas_mz / (1 + alphas_mz * b0 * torch.log(mu * mu / (mz * mz)))
    sgn = torch.tensor([-1.0, -1.0] + [1.0] * m, dtype=torch.float64)
    pphys = (k[..., 1:] * sgn[None, :, None])
    eps = torch.stack([polvec(pphys[:, i], ((hel >> i) & 1).bool()) for i in range(n)], 1)
    amp = bg_amplitude(order, k, eps)
    E = 2 ** n * math.factorial(n - 1) * (amp.real ** 2 + amp.imag ** 2) / 2 ** (n - 2)
    f = lambda xx: 1.7 * xx ** -0.2 * (1 - xx) ** 5
    phi_m = (2 * math.pi) ** (4 - 3 * m) * (math.pi / 2) ** (m - 1) / (math.factorial(m - 1) * math.factorial(m - 2))
    col = 3.0 ** (n - 2) * 8.0 / (256.0 * math.factorial(m))
    w = (lnxmin ** 2 * f(x1) * f(x2) / (2 * shat) * phi_m * shat ** (m - 2) * col
         * (4 * math.pi * alphas) ** (n - 2) * E * GEV2_PB)
    return torch.where(ok, w, torch.zeros_like(w)), dict(alphas=alphas, ht=ht, pass_=ok, k=k, E=E)
