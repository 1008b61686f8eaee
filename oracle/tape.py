"""A small generic reverse-mode tape over numpy float64 arrays.

Test infrastructure only (see ``oracle/__init__.py``).

The paper obtains parameter gradients "by reverse-mode differentiation of the
scalar loss" (Sec. 3.1.1); explicit differentiation replaces only the
coordinate-derivative evaluation.  This tape is that reverse mode in its most
plain form: every primitive (add, sub, mul, neg, matmul, tanh, sum) records
its vector-Jacobian product, and ``backward`` walks the graph in reverse
topological order.  It knows nothing about jets or layers; run over the
hyper-dual program of ``hyperdual.py`` it differentiates through the exact
coordinate derivatives.

Parity: pinned by tests/test_oracle_pins.py (hand-derived width-1 gradient,
central finite differences in every parameter, Taylor remainder of order 2,
agreement with torch float64 autograd).
"""

import numpy as np


def _unbroadcast(g, shape):
    """Sum g over the axes that broadcasting added or stretched to reach g.shape."""
    if g.shape == tuple(shape):
        return g
    while g.ndim > len(shape):
        g = g.sum(axis=0)
    for ax, n in enumerate(shape):
        if n == 1 and g.shape[ax] != 1:
            g = g.sum(axis=ax, keepdims=True)
    return g


class Var:
    __slots__ = ("value", "parents", "grad")
    __array_ufunc__ = None  # make numpy defer to the reflected operators

    def __init__(self, value, parents=()):
        self.value = np.asarray(value, dtype=np.float64)
        self.parents = parents  # tuple of (Var, vjp: g -> contribution)
        self.grad = None

    @staticmethod
    def _wrap(o):
        return o if isinstance(o, Var) else Var(o)

    # --- primitives ---------------------------------------------------------
    def __add__(self, o):
        if not isinstance(o, Var) and hasattr(o, "a"):  # a Dual on the right
            return NotImplemented
        o = Var._wrap(o)
        sa, sb = self.value.shape, o.value.shape
        return Var(self.value + o.value,
                   ((self, lambda g: _unbroadcast(g, sa)),
                    (o, lambda g: _unbroadcast(g, sb))))

    def __radd__(self, o):
        return Var._wrap(o) + self

    def __sub__(self, o):
        if not isinstance(o, Var) and hasattr(o, "a"):
            return NotImplemented
        o = Var._wrap(o)
        sa, sb = self.value.shape, o.value.shape
        return Var(self.value - o.value,
                   ((self, lambda g: _unbroadcast(g, sa)),
                    (o, lambda g: -_unbroadcast(g, sb))))

    def __rsub__(self, o):
        return Var._wrap(o) - self

    def __neg__(self):
        return Var(-self.value, ((self, lambda g: -g),))

    def __mul__(self, o):
        if not isinstance(o, Var) and hasattr(o, "a"):
            return NotImplemented
        o = Var._wrap(o)
        a, b = self.value, o.value
        return Var(a * b,
                   ((self, lambda g: _unbroadcast(g * b, a.shape)),
                    (o, lambda g: _unbroadcast(g * a, b.shape))))

    def __rmul__(self, o):
        return Var._wrap(o) * self

    def __matmul__(self, o):
        o = Var._wrap(o)
        a, b = self.value, o.value
        return Var(a @ b,
                   ((self, lambda g: g @ b.T),
                    (o, lambda g: a.T @ g)))

    def __rmatmul__(self, o):
        return Var._wrap(o) @ self

    @property
    def T(self):
        return Var(self.value.T, ((self, lambda g: g.T),))

    def __getitem__(self, idx):
        shape = self.value.shape

        def vjp(g):
            out = np.zeros(shape)
            np.add.at(out, idx, g)
            return out
        return Var(self.value[idx], ((self, vjp),))

    def tanh(self):
        t = np.tanh(self.value)
        return Var(t, ((self, lambda g: g * (1.0 - t * t)),))

    def sum(self):
        shape = self.value.shape
        return Var(self.value.sum(), ((self, lambda g: np.broadcast_to(g, shape).copy()),))


def backward(out):
    """Accumulate d(out)/d(node) into node.grad for every node reachable from out."""
    order, seen = [], set()
    stack = [(out, False)]
    while stack:
        node, done = stack.pop()
        if done:
            order.append(node)
            continue
        if id(node) in seen:
            continue
        seen.add(id(node))
        stack.append((node, True))
        for p, _ in node.parents:
            if id(p) not in seen:
                stack.append((p, False))
    for node in order:
        node.grad = None
    out.grad = np.ones_like(out.value)
    for node in reversed(order):
        g = node.grad
        if g is None:
            continue
        for p, vjp in node.parents:
            c = vjp(g)
            p.grad = c if p.grad is None else p.grad + c
