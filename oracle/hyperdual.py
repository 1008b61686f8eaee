"""Nested hyper-dual numbers (float64) for exact coordinate derivatives.

Test infrastructure only (see ``oracle/__init__.py``).

A first-order dual number is a + b*eps with eps**2 = 0.  Nesting it n times
(each level has its own nilpotent eps_k) gives a number whose coefficient of
eps_1*eps_2*...*eps_n is the n-th mixed directional derivative of the
function along the n seeded directions, exact up to float64 rounding
(Fike & Alonso, "The development of hyper-dual numbers for exact second-
derivative calculations", AIAA 2011; applied recursively).  The paper's
definition of the quantity being computed is the coordinate derivative of the
network output that enters the residual (Sec. 2.2, residual r_theta =
N(u, d_i u, d_ij u, ...)).

The leaves of a ``Dual`` tree are numpy float64 arrays or ``tape.Var`` nodes,
so the same program also runs under the reverse-mode tape.

Parity: pinned by tests/test_oracle_pins.py (width-1 closed form, tanh
derivative polynomials via sympy, identity activation, central finite
differences, agreement with torch float64 nested autograd).
"""

import numpy as np


class Dual:
    """a + b*eps with eps**2 == 0; a and b are leaves or Duals of one less level."""

    __slots__ = ("a", "b")
    __array_ufunc__ = None  # make numpy defer to the reflected operators

    def __init__(self, a, b):
        self.a = a
        self.b = b

    # --- arithmetic -------------------------------------------------------
    def __add__(self, o):
        if isinstance(o, Dual):
            return Dual(self.a + o.a, self.b + o.b)
        return Dual(self.a + o, self.b)

    def __radd__(self, o):
        return Dual(o + self.a, self.b)

    def __sub__(self, o):
        if isinstance(o, Dual):
            return Dual(self.a - o.a, self.b - o.b)
        return Dual(self.a - o, self.b)

    def __rsub__(self, o):
        return Dual(o - self.a, -self.b)

    def __neg__(self):
        return Dual(-self.a, -self.b)

    def __mul__(self, o):
        if isinstance(o, Dual):
            # (a + b e)(c + d e) = ac + (ad + bc) e
            return Dual(self.a * o.a, self.a * o.b + self.b * o.a)
        return Dual(self.a * o, self.b * o)

    def __rmul__(self, o):
        return Dual(o * self.a, o * self.b)

    def __matmul__(self, m):
        # right-multiplication by a matrix that carries no eps part
        return Dual(self.a @ m, self.b @ m)


def tanh(x):
    """tanh on a Dual tree: tanh(a + b e) = tanh(a) + b (1 - tanh(a)^2) e."""
    if isinstance(x, Dual):
        t = tanh(x.a)
        return Dual(t, x.b * (1.0 - t * t))
    if hasattr(x, "tanh"):
        return x.tanh()
    return np.tanh(x)


def identity(x):
    return x


def _const_like(x, depth):
    """Embed x as a Dual of the given depth with all eps parts zero."""
    if depth == 0:
        return x
    inner = _const_like(x, depth - 1)
    return Dual(inner, _zeros_like_tree(inner))


def _zeros_like_tree(x):
    if isinstance(x, Dual):
        return Dual(_zeros_like_tree(x.a), _zeros_like_tree(x.b))
    return np.zeros_like(np.asarray(x, dtype=np.float64))


def seed_input(X, dirs):
    """Seed input points X [N, d] for the nested derivative along ``dirs``.

    dirs = (i_1, ..., i_n) lists one coordinate index per nesting level; the
    top coefficient of any function of the result is then
    d^n f / (dx_{i_1} ... dx_{i_n}).
    """
    X = np.asarray(X, dtype=np.float64)
    if len(dirs) == 0:
        return X
    inner = seed_input(X, dirs[1:])
    e = np.zeros_like(X)
    e[:, dirs[0]] = 1.0
    return Dual(inner, _const_like(e, len(dirs) - 1))


def top_coefficient(x, depth):
    """Coefficient of eps_1 ... eps_depth (follow the b branch at every level)."""
    for _ in range(depth):
        x = x.b
    return x


def value_part(x, depth):
    for _ in range(depth):
        x = x.a
    return x


def dirs_of(alpha):
    """Multi-index (orders per coordinate) -> tuple of seeded coordinate indices."""
    out = []
    for i, k in enumerate(alpha):
        out.extend([i] * int(k))
    return tuple(out)
