"""Pins of the FP64 oracle against what the paper and mathematics fix.

Every test here runs on the CPU (no GPU marker).  Each pins part of the oracle
against a reference other than the oracle itself:

* hand-derived closed forms of width-1 and width-2 networks (the derivatives
  and the Burgers loss gradient of a width-1 net are written out by hand);
* identity activation: the network is affine, so every derivative of order
  >= 2 vanishes exactly and the first-order ones equal the product of the
  weight matrices;
* tanh derivative polynomials from sympy's symbolic differentiation;
* manufactured exact solutions (Burgers viscous shock, Allen-Cahn kink,
  Kuramoto-Tsuzuki KS wave, Taylor-Green vortex for stream-function NS,
  the Helmholtz sine mode) whose derivatives sympy computes: residual == 0;
* central finite differences in the coordinates and in every parameter
  (Eq. 12) and the Taylor remainder of order 2 (Eq. 13-14);
* torch float64 nested autograd, the paper's AD baseline (Sec. 3.1.1).
"""

import math

import numpy as np
import pytest

import oracle
from oracle import hyperdual as hd
from oracle import residuals as R
from paper_2606_29702_gb300 import workloads as wl


def _rng(seed=0):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------------------
# 1. width-1 network: u = c tanh(wx x + wt t + b) + e
# ---------------------------------------------------------------------------

def _width1(seed=3):
    g = _rng(seed)
    wx, wt, b, c, e = g.uniform(-1.5, 1.5, 5)
    layers = [(np.array([[wx, wt]]), np.array([b])), (np.array([[c]]), np.array([e]))]
    X = np.column_stack([g.uniform(-1, 1, 40), g.uniform(0, 1, 40)])
    return (wx, wt, b, c, e), layers, X


def test_width1_closed_form_derivatives():
    (wx, wt, b, c, e), layers, X = _width1()
    q = wx * X[:, 0] + wt * X[:, 1] + b
    a = np.tanh(q)
    s = 1 - a * a
    expect = {
        (0, 0): c * a + e,
        (1, 0): c * wx * s,
        (0, 1): c * wt * s,
        (2, 0): c * wx ** 2 * (-2 * a * s),
        (1, 1): c * wx * wt * (-2 * a * s),
        (3, 0): c * wx ** 3 * s * (6 * a * a - 2),
        (4, 0): c * wx ** 4 * 8 * a * s * (2 - 3 * a * a),
        (2, 1): c * wx ** 2 * wt * s * (6 * a * a - 2),
    }
    jets = oracle.network_jets(layers, X, list(expect))
    for al, ref in expect.items():
        np.testing.assert_allclose(jets[al][:, 0], ref, rtol=1e-13, atol=1e-13, err_msg=str(al))


def test_width1_hand_gradient_burgers():
    (wx, wt, b, c, e), layers, X = _width1(5)
    nu = 0.05
    x, t = X[:, 0], X[:, 1]
    q = wx * x + wt * t + b
    a = np.tanh(q)
    s = 1 - a * a
    ds = -2 * a * s                     # d s / d q
    das = s * s - 2 * a * a * s         # d (a s) / d q
    u, ux, ut, uxx = c * a + e, c * wx * s, c * wt * s, -2 * c * wx ** 2 * a * s
    r = ut + u * ux - nu * uxx
    # d(u, ux, ut, uxx)/d theta, written out by hand for theta = (wx, wt, b, c, e)
    D = {
        "wx": (c * s * x, c * s + c * wx * ds * x, c * wt * ds * x, -4 * c * wx * a * s - 2 * c * wx ** 2 * das * x),
        "wt": (c * s * t, c * wx * ds * t, c * s + c * wt * ds * t, -2 * c * wx ** 2 * das * t),
        "b": (c * s, c * wx * ds, c * wt * ds, -2 * c * wx ** 2 * das),
        "c": (a, wx * s, wt * s, -2 * wx ** 2 * a * s),
        "e": (np.ones_like(x), 0 * x, 0 * x, 0 * x),
    }
    hand = {}
    for k, (du, dux, dut, duxx) in D.items():
        dr = dut + du * ux + u * dux - nu * duxx
        hand[k] = np.mean(2 * r * dr)
    L, rr, grads = oracle.loss_and_grad(R.burgers(nu), layers, X)
    np.testing.assert_allclose(L, np.mean(r * r), rtol=1e-14)
    np.testing.assert_allclose(rr[:, 0], r, rtol=1e-13, atol=1e-14)
    (gW1, gb1), (gW2, gb2) = grads
    got = {"wx": gW1[0, 0], "wt": gW1[0, 1], "b": gb1[0], "c": gW2[0, 0], "e": gb2[0]}
    for k in hand:
        np.testing.assert_allclose(got[k], hand[k], rtol=1e-12, atol=1e-14, err_msg=k)


# ---------------------------------------------------------------------------
# 2. width-2, two hidden layers: explicit scalar chain rule, nonzero biases
# ---------------------------------------------------------------------------

def test_width2_two_layer_hand_chain():
    g = _rng(11)
    W1, b1 = g.normal(size=(2, 2)), g.normal(size=2)
    W2, b2 = g.normal(size=(2, 2)), g.normal(size=2)
    W3, b3 = g.normal(size=(1, 2)), g.normal(size=1)
    layers = [(W1, b1), (W2, b2), (W3, b3)]
    X = np.column_stack([g.uniform(-1, 1, 25), g.uniform(0, 1, 25)])
    x, t = X[:, 0], X[:, 1]
    # layer 1, unit by unit
    z1 = [W1[i, 0] * x + W1[i, 1] * t + b1[i] for i in range(2)]
    a1 = [np.tanh(v) for v in z1]
    s1 = [1 - v * v for v in a1]
    a1x = [s1[i] * W1[i, 0] for i in range(2)]
    a1t = [s1[i] * W1[i, 1] for i in range(2)]
    a1xx = [-2 * a1[i] * s1[i] * W1[i, 0] ** 2 for i in range(2)]
    a1xt = [-2 * a1[i] * s1[i] * W1[i, 0] * W1[i, 1] for i in range(2)]
    # layer 2
    z2 = [W2[j, 0] * a1[0] + W2[j, 1] * a1[1] + b2[j] for j in range(2)]
    z2x = [W2[j, 0] * a1x[0] + W2[j, 1] * a1x[1] for j in range(2)]
    z2t = [W2[j, 0] * a1t[0] + W2[j, 1] * a1t[1] for j in range(2)]
    z2xx = [W2[j, 0] * a1xx[0] + W2[j, 1] * a1xx[1] for j in range(2)]
    z2xt = [W2[j, 0] * a1xt[0] + W2[j, 1] * a1xt[1] for j in range(2)]
    a2 = [np.tanh(v) for v in z2]
    s2 = [1 - v * v for v in a2]
    a2x = [s2[j] * z2x[j] for j in range(2)]
    a2t = [s2[j] * z2t[j] for j in range(2)]
    a2xx = [-2 * a2[j] * s2[j] * z2x[j] ** 2 + s2[j] * z2xx[j] for j in range(2)]
    a2xt = [-2 * a2[j] * s2[j] * z2x[j] * z2t[j] + s2[j] * z2xt[j] for j in range(2)]
    lin = lambda v: W3[0, 0] * v[0] + W3[0, 1] * v[1]  # noqa: E731
    expect = {(0, 0): lin(a2) + b3[0], (1, 0): lin(a2x), (0, 1): lin(a2t), (2, 0): lin(a2xx), (1, 1): lin(a2xt)}
    jets = oracle.network_jets(layers, X, list(expect))
    for al, ref in expect.items():
        np.testing.assert_allclose(jets[al][:, 0], ref, rtol=1e-12, atol=1e-13, err_msg=str(al))


# ---------------------------------------------------------------------------
# 3. identity activation: the network is affine
# ---------------------------------------------------------------------------

def test_identity_activation_affine():
    widths = [3, 7, 5, 6, 2]
    layers = wl.xavier_layers(widths, 4, bias_std=0.3)
    X = wl.points([(-1, 1)] * 3, 30, 9)
    G = np.eye(3)
    h = np.zeros(3)
    for W, b in layers:
        G = W @ G
        h = W @ h + b
    chans = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0), (0, 1, 2), (3, 0, 0), (4, 0, 0)]
    jets = oracle.network_jets(layers, X, chans, act=hd.identity)
    np.testing.assert_allclose(jets[(0, 0, 0)], X @ G.T + h, rtol=1e-13, atol=1e-13)
    for i in range(3):
        e = [0, 0, 0]
        e[i] = 1
        np.testing.assert_allclose(jets[tuple(e)], np.broadcast_to(G[:, i], (30, 2)), rtol=1e-13, atol=1e-14)
    for al in chans:
        if sum(al) >= 2:
            assert np.all(jets[al] == 0.0), al
    # Burgers residual of an affine net: g_t + u g_x (u_xx = 0)
    lay1 = wl.xavier_layers([2, 6, 6, 1], 8, bias_std=0.2)
    X2 = wl.points([(-1, 1), (0, 1)], 20, 1)
    g1 = np.eye(2)
    h1 = np.zeros(2)[:0]
    g1 = lay1[0][0]
    h1 = lay1[0][1]
    for W, b in lay1[1:]:
        g1, h1 = W @ g1, W @ h1 + b
    u = X2 @ g1[0] + h1[0]
    r = oracle.residual(R.burgers(0.3), lay1, X2, act=hd.identity)[:, 0]
    np.testing.assert_allclose(r, g1[0, 1] + u * g1[0, 0], rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------------------
# 4. tanh derivative polynomials (sympy)
# ---------------------------------------------------------------------------

def test_tanh_derivatives_sympy():
    sp = pytest.importorskip("sympy")
    zs = sp.symbols("z")
    z = np.linspace(-2.5, 2.5, 11)
    layers = [(np.array([[1.0]]), np.array([0.0])), (np.array([[1.0]]), np.array([0.0]))]
    jets = oracle.network_jets(layers, z[:, None], [(n,) for n in range(6)])
    a = np.tanh(z)
    s = 1 - a * a
    closed = [a, s, -2 * a * s, s * (6 * a * a - 2), 8 * a * s * (2 - 3 * a * a), 8 * s * (15 * a ** 4 - 15 * a * a + 2)]
    for n in range(6):
        f = sp.lambdify(zs, sp.diff(sp.tanh(zs), zs, n), "mpmath")
        ref = np.array([float(f(v)) for v in z])
        np.testing.assert_allclose(jets[(n,)][:, 0], ref, rtol=1e-12, atol=1e-12, err_msg="order %d" % n)
        np.testing.assert_allclose(closed[n], ref, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# 5. manufactured exact solutions: the residual assembly gives 0
# ---------------------------------------------------------------------------

def _analytic_jets(sp, syms, exprs, needed, X):
    """{alpha: [N, n_out]} from sympy expressions of the outputs."""
    out = {}
    for al in needed:
        cols = []
        for ex in exprs:
            d = ex
            for v, k in zip(syms, al):
                if k:
                    d = sp.diff(d, v, k)
            f = sp.lambdify(syms, d, "numpy")
            val = np.asarray(f(*[X[:, i] for i in range(len(syms))]), dtype=np.float64)
            cols.append(np.broadcast_to(val, (X.shape[0],)))
        out[tuple(al)] = np.stack(cols, axis=1)
    return out


@pytest.mark.parametrize("case", ["burgers", "allen_cahn", "ks", "helmholtz", "ns_psi", "ns_uvp"])
def test_manufactured_solutions(case):
    sp = pytest.importorskip("sympy")
    g = _rng(21)
    if case == "burgers":
        x, t = sp.symbols("x t")
        nu, A, c = 0.05, 0.7, 0.3
        u = c - A * sp.tanh(A * (x - c * t) / (2 * nu))
        fam, syms, exprs = R.burgers(nu), (x, t), [u]
        X = np.column_stack([g.uniform(-1, 1, 50), g.uniform(0, 1, 50)])
    elif case == "allen_cahn":
        x, t = sp.symbols("x t")
        eps, k = 1e-2, 5.0
        u = sp.tanh(x * sp.sqrt(k / (2 * eps)))
        fam, syms, exprs = R.allen_cahn(eps, k), (x, t), [u]
        X = np.column_stack([g.uniform(-0.2, 0.2, 50), g.uniform(0, 1, 50)])
    elif case == "ks":
        x, t = sp.symbols("x t")
        cc = sp.Rational(1, 3)
        kk = sp.sqrt(sp.Rational(11, 19)) / 2
        T = sp.tanh(kk * (x - cc * t))
        u = cc + sp.Rational(15, 19) * sp.sqrt(sp.Rational(11, 19)) * (-9 * T + 11 * T ** 3)
        fam, syms, exprs = R.kuramoto_sivashinsky(1.0, 1.0, 1.0), (x, t), [u]
        X = np.column_stack([g.uniform(-3, 3, 50), g.uniform(0, 1, 50)])
    elif case == "helmholtz":
        x, y, z = sp.symbols("x y z")
        u = sp.sin(sp.pi * x) * sp.sin(sp.pi * y) * sp.sin(sp.pi * z)
        fam, syms, exprs = R.helmholtz(4 * math.pi), (x, y, z), [u]
        X = g.uniform(-1, 1, (50, 3))
    elif case == "ns_uvp":
        # Kovasznay flow (Kovasznay 1948): an exact steady solution of the
        # incompressible Navier-Stokes equations at Reynolds number Re
        x, y = sp.symbols("x y")
        Re = 100
        lam = sp.Rational(Re, 2) - sp.sqrt(sp.Rational(Re * Re, 4) + 4 * sp.pi ** 2)
        u = 1 - sp.exp(lam * x) * sp.cos(2 * sp.pi * y)
        v = lam / (2 * sp.pi) * sp.exp(lam * x) * sp.sin(2 * sp.pi * y)
        p = (1 - sp.exp(2 * lam * x)) / 2
        fam, syms, exprs = R.navier_stokes_uvp(Re), (x, y), [u, v, p]
        X = np.column_stack([g.uniform(-0.5, 1.0, 50), g.uniform(-0.5, 1.5, 50)])
    else:
        x, y, t = sp.symbols("x y t")
        nu = 0.01
        F = sp.exp(-2 * nu * t)
        psi = sp.sin(x) * sp.sin(y) * F
        p = sp.Rational(1, 4) * (sp.cos(2 * x) + sp.cos(2 * y)) * F ** 2
        fam, syms, exprs = R.navier_stokes_psi(nu), (x, y, t), [psi, p]
        X = g.uniform(0, 1, (50, 3)) * np.array([2 * math.pi, 2 * math.pi, 1.0])
    jets = _analytic_jets(sp, syms, exprs, fam.needed, X)
    comps = fam.components(jets, X, None)
    scale = max(1.0, max(np.abs(v).max() for v in jets.values()))
    for r in comps:
        assert np.abs(np.asarray(r)).max() < 1e-11 * scale ** 2, case
    # and a perturbed field must not satisfy it (the check has teeth)
    bad = {k: v * 1.01 for k, v in jets.items()}
    assert max(np.abs(np.asarray(r)).max() for r in fam.components(bad, X, None)) > 1e-6


# ---------------------------------------------------------------------------
# 6. central finite differences in the coordinates (Eq. 12)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d", [2, 3])
def test_fd_in_coordinates(d):
    layers = wl.xavier_layers([d, 9, 9, 9, 2], 31, bias_std=0.2)
    X = wl.points([(-1, 1)] * d, 20, 2)
    chans = [tuple(int(i == j) * k for j in range(d)) for i in range(d) for k in range(4)]
    chans += [tuple([1] * d), tuple([2] + [1] * (d - 1))]
    chans = sorted(set(chans))
    jets = oracle.network_jets(layers, X, chans)
    h = 1e-4
    for al in chans:
        for i in range(d):
            up = list(al)
            up[i] += 1
            up = tuple(up)
            if up not in jets:
                continue
            Xp, Xm = X.copy(), X.copy()
            Xp[:, i] += h
            Xm[:, i] -= h
            fp = oracle.network_jets(layers, Xp, [al])[al]
            fm = oracle.network_jets(layers, Xm, [al])[al]
            fd = (fp - fm) / (2 * h)
            np.testing.assert_allclose(fd, jets[up], rtol=1e-5, atol=1e-6, err_msg="%s + e%d" % (al, i))


# ---------------------------------------------------------------------------
# 7. finite differences in every parameter and the Taylor remainder (Eq. 12-14)
# ---------------------------------------------------------------------------

FAMS = [
    ("burgers", lambda: R.burgers(0.01 / math.pi), [2, 5, 5, 1]),
    ("ks", lambda: R.kuramoto_sivashinsky(1, 1, 1), [2, 4, 4, 1]),
    ("allen_cahn", lambda: R.allen_cahn(1e-4, 5.0), [2, 4, 3, 1]),
    ("helmholtz", lambda: R.helmholtz(4 * math.pi), [3, 4, 4, 1]),
    ("ns_psi", lambda: R.navier_stokes_psi(0.01), [3, 4, 3, 2]),
    ("ns_uvp", lambda: R.navier_stokes_uvp(100.0), [2, 4, 4, 3]),
]


@pytest.mark.parametrize("name,mk,widths", FAMS, ids=[f[0] for f in FAMS])
def test_fd_in_every_parameter(name, mk, widths):
    fam = mk()
    layers = wl.xavier_layers(widths, 17, bias_std=0.1)
    X = wl.points([(-1, 1)] * widths[0], 12, 5)
    L0, _, grads = oracle.loss_and_grad(fam, layers, X)
    theta = wl.pack(layers)
    gflat = wl.pack(grads)
    h = 1e-6
    fd = np.empty_like(theta)
    for k in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd[k] = (oracle.loss_value(fam, wl.unpack(tp, widths), X) - oracle.loss_value(fam, wl.unpack(tm, widths), X)) / (2 * h)
    scale = np.abs(gflat).max()
    np.testing.assert_allclose(gflat, fd, rtol=2e-5, atol=2e-7 * scale)


@pytest.mark.parametrize("name,mk,widths", FAMS, ids=[f[0] for f in FAMS])
def test_taylor_remainder_second_order(name, mk, widths):
    fam = mk()
    layers = wl.xavier_layers(widths, 23, bias_std=0.1)
    X = wl.points([(-1, 1)] * widths[0], 16, 6)
    L0, _, grads = oracle.loss_and_grad(fam, layers, X)
    theta, g = wl.pack(layers), wl.pack(grads)
    v = _rng(7).standard_normal(theta.size)
    eps = [1e-1 / 2 ** k for k in range(6)]
    rem = []
    for e in eps:
        Le = oracle.loss_value(fam, wl.unpack(theta + e * v, widths), X)
        rem.append(abs(Le - L0 - e * g @ v))
    rates = [math.log2(rem[k] / rem[k + 1]) for k in range(len(rem) - 1)]
    assert np.median(rates) > 1.8, rates
    # a wrong gradient leaves a first-order remainder: rate ~1 at small eps
    small = [1e-4 / 2 ** k for k in range(5)]
    bad = [abs(oracle.loss_value(fam, wl.unpack(theta + e * v, widths), X) - L0 - e * 0.9 * g @ v) for e in small]
    bad_rates = [math.log2(bad[k] / bad[k + 1]) for k in range(len(bad) - 1)]
    assert np.median(bad_rates) < 1.3


# ---------------------------------------------------------------------------
# 8. agreement with torch float64 nested autograd (the paper's AD baseline)
# ---------------------------------------------------------------------------

def _torch_nested(fam_name, coefs, layers, X):
    torch = pytest.importorskip("torch")
    Xt = torch.tensor(X, dtype=torch.float64, requires_grad=True)
    params = []
    for W, b in layers:
        params += [torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True)]
    h = Xt
    n_layers = len(layers)
    for l in range(n_layers):
        h = h @ params[2 * l].T + params[2 * l + 1]
        if l < n_layers - 1:
            h = torch.tanh(h)

    def D(f, *idx):
        for i in idx:
            f = torch.autograd.grad(f.sum(), Xt, create_graph=True)[0][:, i]
        return f
    u = h[:, 0]
    if fam_name == "burgers":
        res = [D(u, 1) + u * D(u, 0) - coefs["nu"] * D(u, 0, 0)]
    elif fam_name == "ks":
        ux = D(u, 0)
        uxx = D(ux, 0)
        res = [D(u, 1) + u * ux + uxx + D(D(uxx, 0), 0)]
    elif fam_name == "ns_uvp":
        uu, vv, p = h[:, 0], h[:, 1], h[:, 2]
        Re = coefs["Re"]
        rc = D(uu, 0) + D(vv, 1)
        ru = uu * D(uu, 0) + vv * D(uu, 1) + D(p, 0) - (D(uu, 0, 0) + D(uu, 1, 1)) / Re
        rv = uu * D(vv, 0) + vv * D(vv, 1) + D(p, 1) - (D(vv, 0, 0) + D(vv, 1, 1)) / Re
        res = [rc, ru, rv]
    else:
        psi, p = h[:, 0], h[:, 1]
        nu = coefs["nu"]
        uu, vv = D(psi, 1), -D(psi, 0)
        ru = D(uu, 2) + uu * D(uu, 0) + vv * D(uu, 1) + D(p, 0) - nu * (D(uu, 0, 0) + D(uu, 1, 1))
        rv = D(vv, 2) + uu * D(vv, 0) + vv * D(vv, 1) + D(p, 1) - nu * (D(vv, 0, 0) + D(vv, 1, 1))
        res = [ru, rv]
    loss = sum((r * r).mean() for r in res)
    grads = torch.autograd.grad(loss, params, allow_unused=True)
    grads = [torch.zeros_like(p) if g is None else g for g, p in zip(grads, params)]
    r = torch.stack(res, 1).detach().numpy()
    return float(loss), r, np.concatenate([g.detach().numpy().ravel() for g in grads])


@pytest.mark.parametrize("fam_name,coefs,widths", [
    ("burgers", dict(nu=0.01 / math.pi), [2, 20, 20, 20, 20, 1]),
    ("ks", dict(c1=1.0, c2=1.0, c4=1.0), [2, 16, 16, 16, 1]),
    ("ns_psi", dict(nu=0.01), [3, 12, 12, 12, 2]),
    ("ns_uvp", dict(Re=100.0), [2, 16, 16, 16, 3]),
])
def test_agrees_with_torch_nested_autograd(fam_name, coefs, widths):
    layers = wl.xavier_layers(widths, 1, bias_std=0.1)
    X = wl.points([(-1, 1)] * widths[0], 64, 0)
    fam = R.by_name(fam_name, **coefs)
    L, r, grads = oracle.loss_and_grad(fam, layers, X)
    Lt, rt, gt = _torch_nested(fam_name, coefs, layers, X)
    g = wl.pack(grads)
    assert np.linalg.norm(r - rt) <= 1e-12 * np.linalg.norm(rt)
    assert np.linalg.norm(g - gt) <= 1e-12 * np.linalg.norm(gt)
    assert abs(L - Lt) <= 1e-12 * abs(Lt)


# ---------------------------------------------------------------------------
# 9. generic monomial residual equals the named families
# ---------------------------------------------------------------------------

def test_monomial_family_matches_burgers():
    nu = 0.02
    comps = [[(1.0, [(0, (0, 1))]), (1.0, [(0, (0, 0)), (0, (1, 0))]), (-nu, [(0, (2, 0))])]]
    fam_m = R.monomial_family(2, 1, comps)
    layers = wl.xavier_layers([2, 6, 6, 1], 3, bias_std=0.1)
    X = wl.points([(-1, 1), (0, 1)], 30, 4)
    np.testing.assert_allclose(oracle.residual(fam_m, layers, X), oracle.residual(R.burgers(nu), layers, X), rtol=1e-15, atol=0)


# ---------------------------------------------------------------------------
# 10. Adam against a hand-unrolled update and torch.optim.Adam
# ---------------------------------------------------------------------------

def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    g = _rng(2)
    theta = g.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    p = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-3)
    for step in range(1, 6):
        grad = g.standard_normal(50)
        theta, m, v = oracle.adam_step(theta, m, v, grad, step)
        p.grad = torch.tensor(grad)
        opt.step()
    np.testing.assert_allclose(theta, p.detach().numpy(), rtol=1e-13, atol=1e-15)
    # first step of Adam moves every coordinate by lr * sign(g) (up to eps)
    t1, _, _ = oracle.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), np.array([2.0, -3.0, 0.5]), 1)
    np.testing.assert_allclose(t1, -1e-3 * np.sign([2.0, -3.0, 0.5]), rtol=1e-7)
