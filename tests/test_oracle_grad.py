"""Pins for the FP64 gradient oracle (oracle/grad_torch.py).

It restates the event weight in PyTorch CPU float64 so that autograd gives
exact derivatives.  Pinned against: the C oracle's weights (an independent
implementation of the same function), central finite differences of the C
oracle, the closed form d w / d ln mu_R = -2 (n-2) b0 alpha_s w of one-loop
running, and Euler's theorem for the momentum gradient (|A|^2 is homogeneous
of degree 8 - 2n in the momenta, H_T of degree 1).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import grad_torch as gt  # noqa: E402


def _inputs(orc, n, seed, count, first=0):
    op = orc.process(n)
    ev = [orc.event(op, seed, first + i) for i in range(count)]
    nu = 2 + 4 * (n - 2)
    u = torch.tensor(np.array([orc.uniforms(op, seed, first + i)[:nu] for i in range(count)]))
    hel = torch.tensor([e["hel_bits"] for e in ev])
    order = torch.tensor(np.array([e["perm"] for e in ev]))
    return op, ev, u, hel, order


@pytest.mark.parametrize("n", [4, 6, 8])
def test_torch_weight_equals_c_oracle(orc, n):
    op, ev, u, hel, order = _inputs(orc, n, 5, 60)
    w, _ = gt.weight(u, hel, order, n)
    w = w.numpy()
    ref = np.array([e["weight"] for e in ev])
    # a cut flag may differ where a cut quantity sits at its threshold (torch
    # and libm transcendentals differ by an ulp): at most one such event
    same = (w > 0) == (ref > 0)
    assert (~same).sum() <= 1
    ok = same & (ref > 0)
    assert np.all(w[same & (ref == 0)] == 0)
    # vanishing helicity amplitudes are rounding noise: absolute scale from the largest weight
    assert np.all(np.abs(w[ok] - ref[ok]) <= 1e-10 * ref[ok] + 1e-12 * ref.max())


@pytest.mark.parametrize("n", [4, 6])
def test_autograd_matches_c_oracle_finite_differences(orc, n):
    op, ev, u, hel, order = _inputs(orc, n, 9, 200)
    uu = u.clone().requires_grad_(True)
    w, _ = gt.weight(uu, hel, order, n)
    (g,) = torch.autograd.grad(w.sum(), uu)
    checked = 0
    wmax = max(x["weight"] for x in ev)
    for i, e in enumerate(ev):
        c = bin(e["hel_bits"]).count("1")
        if not e["pass"] or c <= 1 or c >= n - 1 or e["weight"] < 1e-6 * wmax:
            continue  # vanishing helicity amplitudes are rounding noise
        u0 = orc.uniforms(op, 9, i)
        for j in range(u.shape[1]):
            h = 1e-6 * min(u0[j], 1 - u0[j])
            up, um = u0.copy(), u0.copy()
            up[j] += h
            um[j] -= h
            a, b = orc.event_u(op, up), orc.event_u(op, um)
            if not (a["pass"] and b["pass"]):
                continue
            fd = (a["weight"] - b["weight"]) / (2 * h)
            gn = float(g[i].abs().max())
            assert abs(fd - float(g[i, j])) <= 1e-5 * gn, (i, j, fd, float(g[i, j]))
            checked += 1
    assert checked > 40


@pytest.mark.parametrize("n", [5, 7])
def test_log_mu_derivative_closed_form(orc, n):
    op, ev, u, hel, order = _inputs(orc, n, 3, 40)
    lx = torch.zeros((), dtype=torch.float64, requires_grad=True)
    w, aux = gt.weight(u, hel, order, n, mu_r_factor=0.5 * torch.exp(lx))
    (g,) = torch.autograd.grad(w.sum(), lx)
    b0 = 23 / (12 * math.pi)
    closed = float((-2 * (n - 2) * b0 * aux["alphas"] * w).sum())
    assert math.isclose(g.item(), closed, rel_tol=1e-10)


@pytest.mark.parametrize("n", [4, 6, 8])
def test_momentum_gradient_euler_identity(orc, n):
    # scaling every momentum by lambda at fixed x: |A|^2 -> lambda^(8-2n), H_T -> lambda H_T
    op, ev, u, hel, order = _inputs(orc, n, 4, 40)
    _, _, _, k, _ = gt.kinematics(u, n)
    kk = k.clone().requires_grad_(True)
    w, aux = gt.weight(u, hel, order, n, k_override=kk)
    (g,) = torch.autograd.grad(w.sum(), kk)
    b0 = 23 / (12 * math.pi)
    lhs = (g * k).sum((1, 2))
    rhs = w * ((8 - 2 * n) - 2 * (n - 2) * b0 * aux["alphas"])
    ok = w > 0
    # vanishing helicity amplitudes are rounding noise: absolute scale from the largest weight
    assert torch.allclose(lhs[ok], rhs[ok], rtol=1e-8, atol=1e-10 * float(w.max()))
