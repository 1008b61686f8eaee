"""Composite PINN losses with all-points batching, written out plainly.

Test infrastructure only (see ``oracle/__init__.py``).

Sec. 3.1.1 trains on a loss that sums weighted terms -- initial-condition,
boundary-condition and PDE-residual terms -- each over its own point set, and
evaluates the network once on all points: the point sets are concatenated
before the network evaluation and the outputs are split afterwards to
assemble the terms.  Here:

    L = sum_g  w_g * (1 / M_g) * sum_{m < M_g} sum_c r_{g,c,m}^2

where term g owns a contiguous block of the concatenated points.  A plain term
has one residual per point (M_g = its point count).  A paired term owns its
points as consecutive pairs (a_m, b_m) and has one residual per pair, built
from the output jets at both points (M_g = half its point count): the
periodic boundary conditions u(0, t) = u(1, t) and u_x(0, t) = u_x(1, t) of
the Burgers case are such terms.

Terms are given as ``Term(fn, needed, weight, paired, n_res)``: ``fn(U, Ub, X,
src)`` returns the list of residual components from the output jets of the
term's (first) points ``U[(o, alpha)]``, the jets of the second points of the
pairs ``Ub`` (None for a plain term), the term's points and its source rows.

The coordinate derivatives come from ``pinn.network_jets`` (nested hyper-dual
numbers) on the concatenated points, and the gradient from the reverse tape,
exactly as for a single residual.

Parity: pinned by tests/test_oracle_losses.py (hand-written special cases,
the sum of separately evaluated terms, central finite differences in every
parameter, agreement with torch nested autograd).
"""

import numpy as np

from . import hyperdual as hd
from .pinn import network_jets
from .tape import Var, backward


class Term:
    def __init__(self, fn, needed, weight=1.0, paired=False, n_res=1, name="term"):
        self.fn = fn
        self.needed = [tuple(a) for a in needed]
        self.weight = float(weight)
        self.paired = bool(paired)
        self.n_res = int(n_res)
        self.name = name


def _split(jets, lo, hi, n_out, step=1, offset=0):
    U = {}
    for alpha, arr in jets.items():
        for o in range(n_out):
            U[(o, alpha)] = arr[lo + offset:hi:step, o]
    return U


def _assemble(terms, counts, jets, X, sources, n_out):
    """Residual components and their mean-square weights, term by term."""
    out = []
    lo = 0
    for g, (t, cnt) in enumerate(zip(terms, counts)):
        hi = lo + cnt
        src = None if sources is None else sources[g]
        if t.paired:
            if cnt % 2:
                raise ValueError("a paired term needs an even number of points")
            Ua = _split(jets, lo, hi, n_out, 2, 0)
            Ub = _split(jets, lo, hi, n_out, 2, 1)
            comps = t.fn(Ua, Ub, X[lo:hi:2], src)
            M = cnt // 2
        else:
            Ua = _split(jets, lo, hi, n_out)
            comps = t.fn(Ua, None, X[lo:hi], src)
            M = cnt
        out.append((comps, t.weight / M if M else 0.0, M))
        lo = hi
    return out


def _channels(terms, d):
    chans = {tuple([0] * d)}
    for t in terms:
        chans |= set(t.needed)
    return sorted(chans)


def residuals(terms, counts, layers, X, sources=None, act=hd.tanh):
    """Per-term residual arrays [M_g, n_res_g] on the concatenated points X."""
    X = np.asarray(X, dtype=np.float64)
    n_out = np.asarray(layers[-1][0]).shape[0]
    jets = network_jets(layers, X, _channels(terms, X.shape[1]), act)
    res = []
    for comps, _, M in _assemble(terms, counts, jets, X, sources, n_out):
        res.append(np.stack([np.broadcast_to(np.asarray(c.value if isinstance(c, Var) else c, dtype=np.float64),
                                             (M,)) for c in comps], axis=1))
    return res


def loss_value(terms, counts, layers, X, sources=None, act=hd.tanh):
    X = np.asarray(X, dtype=np.float64)
    n_out = np.asarray(layers[-1][0]).shape[0]
    jets = network_jets(layers, X, _channels(terms, X.shape[1]), act)
    total = 0.0
    for comps, scale, _ in _assemble(terms, counts, jets, X, sources, n_out):
        for c in comps:
            c = np.asarray(c, dtype=np.float64)
            total += scale * float((c * c).sum())
    return total


def loss_and_grad(terms, counts, layers, X, sources=None, act=hd.tanh):
    """(L, [r_g], grads) with grads a list of (dL/dW, dL/db) per layer."""
    X = np.asarray(X, dtype=np.float64)
    if sum(counts) != X.shape[0]:
        raise ValueError("the term point counts must add up to the number of points")
    n_out = np.asarray(layers[-1][0]).shape[0]
    vlayers = [(Var(np.array(W, dtype=np.float64)), Var(np.array(b, dtype=np.float64))) for W, b in layers]
    jets = network_jets(vlayers, X, _channels(terms, X.shape[1]), act)
    loss = None
    res = []
    for comps, scale, M in _assemble(terms, counts, jets, X, sources, n_out):
        vals = []
        for c in comps:
            if not isinstance(c, Var):
                raise TypeError("a loss component does not depend on the parameters")
            term = (c * c).sum() * scale
            loss = term if loss is None else loss + term
            vals.append(c.value)
        res.append(np.stack(vals, axis=1))
    backward(loss)
    grads = []
    for W, b in vlayers:
        gW = W.grad if W.grad is not None else np.zeros_like(W.value)
        gb = b.grad if b.grad is not None else np.zeros_like(b.value)
        grads.append((gW, gb))
    return float(loss.value), res, grads


# ---------------------------------------------------------------------------
# The two composite losses of Sec. 3.1.1 (the terms besides the PDE residual)
# ---------------------------------------------------------------------------

def burgers_terms(nu, w_ic=1.0, w_bc=1.0, w_pde=1.0):
    """Burgers on (x, t) in [0, 1] x [0, 1] (Sec. 3.1.1): periodic boundary
    terms for u and u_x (pairs (0, t_m), (1, t_m)), an initial-condition term
    u(x, 0) - u0(x) with u0 given per point as the source, and the PDE
    residual u_t + u u_x - nu u_xx."""
    O, DX, DT, DXX = (0, 0), (1, 0), (0, 1), (2, 0)

    def bc(U, Ub, X, src):
        return [U[(0, O)] - Ub[(0, O)], U[(0, DX)] - Ub[(0, DX)]]

    def ic(U, Ub, X, src):
        return [U[(0, O)] - np.asarray(src, dtype=np.float64).reshape(-1)]

    def pde(U, Ub, X, src):
        u = U[(0, O)]
        return [U[(0, DT)] + u * U[(0, DX)] - nu * U[(0, DXX)]]

    return [Term(bc, [O, DX], w_bc, True, 2, "periodic_bc"),
            Term(ic, [O], w_ic, False, 1, "ic"),
            Term(pde, [O, DX, DT, DXX], w_pde, False, 1, "pde")]


def cavity_terms(Re=100.0, w_wall=1.0, w_lid=1.0, w_pde=1.0):
    """Lid-driven cavity on [0, 1]^2 (Sec. 3.1.1): the three residuals of
    Eq. 16, the no-slip walls u = v = 0 and the lid (y = 1) u = 1, v = 0; the
    prescribed velocities come per point as the source."""
    O, DX, DY, DXX, DYY = (0, 0), (1, 0), (0, 1), (2, 0), (0, 2)

    def pde(U, Ub, X, src):
        u, v = U[(0, O)], U[(1, O)]
        ux, uy, vx, vy = U[(0, DX)], U[(0, DY)], U[(1, DX)], U[(1, DY)]
        return [ux + vy,
                u * ux + v * uy + U[(2, DX)] - (U[(0, DXX)] + U[(0, DYY)]) * (1.0 / Re),
                u * vx + v * vy + U[(2, DY)] - (U[(1, DXX)] + U[(1, DYY)]) * (1.0 / Re)]

    def velocity(U, Ub, X, src):
        s = np.asarray(src, dtype=np.float64).reshape(X.shape[0], -1)
        return [U[(0, O)] - s[:, 0], U[(1, O)] - s[:, 1]]

    return [Term(pde, [O, DX, DY, DXX, DYY], w_pde, False, 3, "pde"),
            Term(velocity, [O], w_wall, False, 2, "wall"),
            Term(velocity, [O], w_lid, False, 2, "lid")]
