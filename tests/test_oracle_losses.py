"""Pins of the composite-loss oracle (oracle/losses.py): the all-points-batched
loss of Sec. 3.1.1, checked against what fixes it independently of its code.

* additivity: the composite loss and gradient equal the weighted sum of the
  terms evaluated one at a time on their own points (the single-residual
  oracle for the PDE term), so the concatenation, the splitting of the
  outputs, the pairing and the per-term means are right;
* pairing: a periodic-boundary pair whose two points coincide has residual
  exactly 0, and swapping the two points of every pair leaves the loss
  unchanged but flips the residual's sign;
* central finite differences of the composite loss in every parameter;
* agreement with torch float64 nested autograd on the same composite loss.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import losses as Lo
from oracle import residuals as R
from paper_2606_29702_gb300 import workloads as wl


def _burgers_case(n_bc=6, n_ic=5, n_pde=9, seed=0, widths=(2, 6, 6, 1)):
    g = np.random.default_rng(seed)
    t = g.random(n_bc)
    bc = np.empty((2 * n_bc, 2))
    bc[0::2, 0], bc[1::2, 0] = 0.0, 1.0
    bc[0::2, 1] = bc[1::2, 1] = t
    ic = np.column_stack([g.random(n_ic), np.zeros(n_ic)])
    pde = g.random((n_pde, 2))
    X = np.concatenate([bc, ic, pde])
    counts = [2 * n_bc, n_ic, n_pde]
    sources = [None, np.sin(2 * math.pi * ic[:, 0]), None]
    layers = wl.xavier_layers(list(widths), seed + 3, bias_std=0.2)
    return X, counts, sources, layers


def test_burgers_composite_equals_sum_of_terms():
    nu = 0.02
    X, counts, sources, layers = _burgers_case()
    terms = Lo.burgers_terms(nu, w_ic=3.0, w_bc=0.5, w_pde=2.0)
    L, res, grads = Lo.loss_and_grad(terms, counts, layers, X, sources)
    nb, ni, npde = counts
    # PDE term alone: the single-residual oracle on its points, times its weight
    Lp, rp, gp = oracle.loss_and_grad(R.burgers(nu), layers, X[nb + ni:])
    # IC term alone: u - u0 as a monomial family with a source column
    fam_ic = R.monomial_family(2, 1, [[(1.0, [(0, (0, 0))])]], has_source=True)
    Li, ri, gi = oracle.loss_and_grad(fam_ic, layers, X[nb:nb + ni], source=sources[1][:, None])
    # periodic term alone, from the network jets at both points of every pair
    jets = oracle.network_jets(layers, X[:nb], [(0, 0), (1, 0)])
    rb = np.stack([jets[(0, 0)][0::2, 0] - jets[(0, 0)][1::2, 0], jets[(1, 0)][0::2, 0] - jets[(1, 0)][1::2, 0]], 1)
    Lb = float((rb ** 2).sum() / (nb // 2))
    assert abs(L - (0.5 * Lb + 3.0 * Li + 2.0 * Lp)) <= 1e-13 * abs(L)
    np.testing.assert_allclose(res[0], rb, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(res[1], ri, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(res[2], rp, rtol=1e-13, atol=1e-15)
    # the gradient is the same linear combination (the periodic term's own
    # gradient from the composite oracle on its points alone, weight included)
    Lbc, _, gbc = Lo.loss_and_grad([terms[0]], [nb], layers, X[:nb])
    assert abs(Lbc - 0.5 * Lb) <= 1e-13 * abs(Lb)
    g = wl.pack(grads)
    comb = wl.pack(gbc) + 3.0 * wl.pack(gi) + 2.0 * wl.pack(gp)
    np.testing.assert_allclose(g, comb, rtol=1e-12, atol=1e-14 * np.abs(g).max())


def test_pairing_special_cases():
    X, counts, sources, layers = _burgers_case()
    nb = counts[0]
    terms = [Lo.burgers_terms(0.02)[0]]
    same = X[:nb].copy()
    same[1::2] = same[0::2]  # both points of every pair coincide
    L0, r0, g0 = Lo.loss_and_grad(terms, [nb], layers, same)
    assert L0 == 0.0 and np.all(r0[0] == 0.0)
    assert all(np.all(gW == 0) and np.all(gb == 0) for gW, gb in g0)
    swapped = X[:nb].copy()
    swapped[0::2], swapped[1::2] = X[1:nb:2], X[0:nb:2]
    La, ra, _ = Lo.loss_and_grad(terms, [nb], layers, X[:nb])
    Lb, rb, _ = Lo.loss_and_grad(terms, [nb], layers, swapped)
    assert abs(La - Lb) <= 1e-14 * La and La > 0
    np.testing.assert_allclose(rb[0], -ra[0], rtol=0, atol=1e-15)


@pytest.mark.parametrize("which", ["burgers", "cavity"])
def test_composite_fd_in_every_parameter(which):
    if which == "burgers":
        X, counts, sources, layers = _burgers_case(n_bc=3, n_ic=3, n_pde=4, widths=(2, 4, 3, 1))
        terms = Lo.burgers_terms(0.05, w_ic=2.0, w_bc=0.7)
    else:
        X, counts, sources, layers = _cavity_case(n_pde=4, n_wall=3, n_lid=3, widths=(2, 4, 3, 3))
        terms = Lo.cavity_terms(100.0, w_wall=1.5, w_lid=0.5)
    widths = [layers[0][0].shape[1]] + [W.shape[0] for W, _ in layers]
    L0, _, grads = Lo.loss_and_grad(terms, counts, layers, X, sources)
    theta = wl.pack(layers)
    g = wl.pack(grads)
    h = 1e-6
    fd = np.empty_like(theta)
    for k in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd[k] = (Lo.loss_value(terms, counts, wl.unpack(tp, widths), X, sources)
                 - Lo.loss_value(terms, counts, wl.unpack(tm, widths), X, sources)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=2e-5, atol=2e-7 * np.abs(g).max())


def _cavity_case(n_pde=9, n_wall=7, n_lid=5, seed=1, widths=(2, 6, 6, 3)):
    g = np.random.default_rng(seed)
    pde = g.random((n_pde, 2))
    s = g.random(n_wall)
    side = g.integers(0, 3, n_wall)
    wall = np.where(side[:, None] == 0, np.column_stack([np.zeros(n_wall), s]),
                    np.where(side[:, None] == 1, np.column_stack([np.ones(n_wall), s]),
                             np.column_stack([s, np.zeros(n_wall)])))
    lid = np.column_stack([g.random(n_lid), np.ones(n_lid)])
    X = np.concatenate([pde, wall, lid])
    counts = [n_pde, n_wall, n_lid]
    sources = [None, np.zeros((n_wall, 2)), np.column_stack([np.ones(n_lid), np.zeros(n_lid)])]
    layers = wl.xavier_layers(list(widths), seed + 5, bias_std=0.2)
    return X, counts, sources, layers


def _torch_composite(which, layers, X, counts, sources, coefs):
    torch = pytest.importorskip("torch")
    Xt = torch.tensor(X, dtype=torch.float64, requires_grad=True)
    params = []
    for W, b in layers:
        params += [torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True)]
    h = Xt
    for l in range(len(layers)):
        h = h @ params[2 * l].T + params[2 * l + 1]
        if l < len(layers) - 1:
            h = torch.tanh(h)

    def D(f, *idx):
        for i in idx:
            f = torch.autograd.grad(f.sum(), Xt, create_graph=True)[0][:, i]
        return f
    if which == "burgers":
        nb, ni, npde = counts
        u = h[:, 0]
        ux = D(u, 0)
        rbc = [u[0:nb:2] - u[1:nb:2], ux[0:nb:2] - ux[1:nb:2]]
        ric = [u[nb:nb + ni] - torch.tensor(sources[1])]
        s = slice(nb + ni, nb + ni + npde)
        rp = [D(u, 1)[s] + u[s] * ux[s] - coefs["nu"] * D(ux, 0)[s]]
        parts = [(rbc, coefs["w_bc"], nb // 2), (ric, coefs["w_ic"], ni), (rp, 1.0, npde)]
    else:
        npde, nw, nl = counts
        u, v, p = h[:, 0], h[:, 1], h[:, 2]
        Re = coefs["Re"]
        s = slice(0, npde)
        ux, uy, vx, vy = D(u, 0), D(u, 1), D(v, 0), D(v, 1)
        lu, lv = D(ux, 0) + D(uy, 1), D(vx, 0) + D(vy, 1)
        rp = [(ux + vy)[s], (u * ux + v * uy + D(p, 0) - lu / Re)[s], (u * vx + v * vy + D(p, 1) - lv / Re)[s]]
        sw, sl = slice(npde, npde + nw), slice(npde + nw, npde + nw + nl)
        lid = torch.tensor(sources[2])
        parts = [(rp, 1.0, npde), ([u[sw], v[sw]], coefs["w_wall"], nw),
                 ([u[sl] - lid[:, 0], v[sl] - lid[:, 1]], coefs["w_lid"], nl)]
    loss = sum(w / M * sum((r * r).sum() for r in rs) for rs, w, M in parts)
    grads = torch.autograd.grad(loss, params)
    return float(loss), np.concatenate([gg.detach().numpy().ravel() for gg in grads])


@pytest.mark.parametrize("which", ["burgers", "cavity"])
def test_composite_agrees_with_torch_nested_autograd(which):
    if which == "burgers":
        X, counts, sources, layers = _burgers_case(n_bc=10, n_ic=7, n_pde=20, widths=(2, 12, 12, 12, 1))
        coefs = dict(nu=0.01, w_ic=4.0, w_bc=0.25)
        terms = Lo.burgers_terms(coefs["nu"], w_ic=coefs["w_ic"], w_bc=coefs["w_bc"])
    else:
        X, counts, sources, layers = _cavity_case(n_pde=20, n_wall=11, n_lid=7, widths=(2, 12, 12, 12, 3))
        coefs = dict(Re=100.0, w_wall=2.0, w_lid=0.5)
        terms = Lo.cavity_terms(coefs["Re"], w_wall=coefs["w_wall"], w_lid=coefs["w_lid"])
    L, _, grads = Lo.loss_and_grad(terms, counts, layers, X, sources)
    Lt, gt = _torch_composite(which, layers, X, counts, sources, coefs)
    g = wl.pack(grads)
    assert abs(L - Lt) <= 1e-12 * abs(Lt)
    assert np.linalg.norm(g - gt) <= 1e-12 * np.linalg.norm(gt)
