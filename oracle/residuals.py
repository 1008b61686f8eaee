"""PDE residual families, written out as plain formulas.

Test infrastructure only (see ``oracle/__init__.py``).

Each family names the multi-indices its residual uses (``needed``; a
multi-index is the tuple of derivative orders per input coordinate) and
assembles r = N(u, du, ...) from the network's coordinate derivatives
(Sec. 2.2: r_theta(x) = N(u_theta, d_i u_theta, d_ij u_theta, ...)).

Families and the passages they follow:
* Burgers, r = u_t + u u_x - nu u_xx, inputs (x, t) (Sec. 3.1.1; the viscosity
  is a parameter: the paper uses 0.01, the 2->20x4->1 workload uses 0.01/pi).
* Kuramoto-Sivashinsky, r = u_t + c1 u u_x + c2 u_xx + c4 u_xxxx, inputs
  (x, t) (Sec. 3.1.1 with coefficients 5, 0.5, 0.005; the 2->64x5->1 workload
  uses 1, 1, 1).
* Allen-Cahn, r = u_t - eps u_xx + k u^3 - k u, inputs (x, t) (eps = 1e-4,
  k = 5 in the ensemble workload; not in the paper's experiments).
* Helmholtz, r = u_xx + u_yy + u_zz + k^2 u - f, inputs (x, y, z), with
  f = (k^2 - 3 pi^2) sin(pi x) sin(pi y) sin(pi z) manufactured from
  u = sin(pi x) sin(pi y) sin(pi z) (3-D Helmholtz workload).
* Navier-Stokes in stream-function form, inputs (x, y, t), outputs (psi, p),
  u = psi_y, v = -psi_x: the two momentum residuals of Eq. 16 with the time
  derivative kept (t is an input) and nu = 1/Re:
      r_u = u_t + u u_x + v u_y + p_x - nu (u_xx + u_yy)
      r_v = v_t + u v_x + v v_y + p_y - nu (v_xx + v_yy)
  The continuity residual of Eq. 16 vanishes identically for u = psi_y,
  v = -psi_x and is not assembled.
* Navier-Stokes in primitive variables, Eq. 16 as printed: inputs (x, y),
  outputs (u, v, p), steady, Re = 100 in the lid-driven cavity of Sec. 3.1.1:
      r_c = u_x + v_y
      r_u = u u_x + v u_y + p_x - (u_xx + u_yy) / Re
      r_v = u v_x + v v_y + p_y - (v_xx + v_yy) / Re
* Generic: a list of components, each a sum of monomials coef * prod_j
  d^{alpha_j} u_{o_j}, minus an optional per-point source column.

Parity: pinned by tests/test_oracle_pins.py (manufactured solutions whose
derivatives sympy computes symbolically make every residual vanish).
"""

import math

import numpy as np


class Family:
    def __init__(self, name, d_in, n_out, needed, fn):
        self.name = name
        self.d_in = d_in
        self.n_out = n_out
        self.needed = [tuple(a) for a in needed]
        self._fn = fn

    def components(self, jets, X, source=None):
        U = {}
        for alpha, arr in jets.items():
            for o in range(self.n_out):
                U[(o, alpha)] = arr[:, o]
        return self._fn(U, X, source)


def burgers(nu):
    X_, T_ = (1, 0), (0, 1)
    need = [(0, 0), T_, X_, (2, 0)]

    def fn(U, X, source):
        u, ut, ux, uxx = U[(0, (0, 0))], U[(0, T_)], U[(0, X_)], U[(0, (2, 0))]
        return [ut + u * ux - nu * uxx]
    return Family("burgers", 2, 1, need, fn)


def kuramoto_sivashinsky(c1=1.0, c2=1.0, c4=1.0):
    need = [(0, 0), (0, 1), (1, 0), (2, 0), (4, 0)]

    def fn(U, X, source):
        u, ut, ux = U[(0, (0, 0))], U[(0, (0, 1))], U[(0, (1, 0))]
        uxx, uxxxx = U[(0, (2, 0))], U[(0, (4, 0))]
        return [ut + c1 * u * ux + c2 * uxx + c4 * uxxxx]
    return Family("ks", 2, 1, need, fn)


def allen_cahn(eps=1e-4, k=5.0):
    need = [(0, 0), (0, 1), (2, 0)]

    def fn(U, X, source):
        u, ut, uxx = U[(0, (0, 0))], U[(0, (0, 1))], U[(0, (2, 0))]
        return [ut - eps * uxx + k * u * u * u - k * u]
    return Family("allen_cahn", 2, 1, need, fn)


def helmholtz_source(X, k):
    X = np.asarray(X, dtype=np.float64)
    pi = math.pi
    return (k * k - 3.0 * pi * pi) * np.sin(pi * X[:, 0]) * np.sin(pi * X[:, 1]) * np.sin(pi * X[:, 2])


def helmholtz(k=4.0 * math.pi):
    need = [(0, 0, 0), (2, 0, 0), (0, 2, 0), (0, 0, 2)]

    def fn(U, X, source):
        u = U[(0, (0, 0, 0))]
        f = helmholtz_source(X, k) if source is None else np.asarray(source, dtype=np.float64).reshape(-1)
        return [U[(0, (2, 0, 0))] + U[(0, (0, 2, 0))] + U[(0, (0, 0, 2))] + k * k * u - f]
    return Family("helmholtz", 3, 1, need, fn)


def navier_stokes_psi(nu=0.01):
    # inputs (x, y, t); outputs 0 = psi, 1 = p
    def a(x=0, y=0, t=0):
        return (x, y, t)
    need = [a(), a(x=1), a(y=1), a(t=1), a(x=2), a(x=1, y=1), a(y=2), a(x=1, t=1), a(y=1, t=1),
            a(x=3), a(x=2, y=1), a(x=1, y=2), a(y=3)]

    def fn(U, X, source):
        P = lambda **kw: U[(0, a(**kw))]  # noqa: E731  psi derivatives
        p_x, p_y = U[(1, a(x=1))], U[(1, a(y=1))]
        u, v = P(y=1), -P(x=1)
        u_t, v_t = P(y=1, t=1), -P(x=1, t=1)
        u_x, u_y = P(x=1, y=1), P(y=2)
        v_x, v_y = -P(x=2), -P(x=1, y=1)
        lap_u = P(x=2, y=1) + P(y=3)
        lap_v = -(P(x=3) + P(x=1, y=2))
        r_u = u_t + u * u_x + v * u_y + p_x - nu * lap_u
        r_v = v_t + u * v_x + v * v_y + p_y - nu * lap_v
        return [r_u, r_v]
    fam = Family("ns_psi", 3, 2, need, fn)
    return fam


def navier_stokes_uvp(Re=100.0):
    # inputs (x, y); outputs 0 = u, 1 = v, 2 = p
    O, DX, DY, DXX, DYY = (0, 0), (1, 0), (0, 1), (2, 0), (0, 2)
    need = [O, DX, DY, DXX, DYY]

    def fn(U, X, source):
        u, v = U[(0, O)], U[(1, O)]
        u_x, u_y, v_x, v_y = U[(0, DX)], U[(0, DY)], U[(1, DX)], U[(1, DY)]
        p_x, p_y = U[(2, DX)], U[(2, DY)]
        lap_u = U[(0, DXX)] + U[(0, DYY)]
        lap_v = U[(1, DXX)] + U[(1, DYY)]
        r_c = u_x + v_y
        r_u = u * u_x + v * u_y + p_x - lap_u * (1.0 / Re)
        r_v = u * v_x + v * v_y + p_y - lap_v * (1.0 / Re)
        return [r_c, r_u, r_v]
    return Family("ns_uvp", 2, 3, need, fn)


def monomial_family(d_in, n_out, components, has_source=False):
    """Generic residual: components[c] = list of (coef, [(o, alpha), ...]).

    r_c(x_n) = sum_m coef_m prod_j d^{alpha_j} u_{o_j}(x_n) - s_c(x_n), where the
    optional source s [N, n_res] is supplied by the caller.
    """
    need = sorted({tuple(al) for comp in components for _, facs in comp for _, al in facs} | {tuple([0] * d_in)})

    def fn(U, X, source):
        out = []
        for c, comp in enumerate(components):
            acc = None
            for coef, facs in comp:
                term = coef
                for o, al in facs:
                    term = term * U[(o, tuple(al))]
                acc = term if acc is None else acc + term
            if has_source and source is not None:
                acc = acc - np.asarray(source, dtype=np.float64).reshape(X.shape[0], -1)[:, c]
            out.append(acc)
        return out
    return Family("monomial", d_in, n_out, need, fn)


def by_name(name, **kw):
    table = {
        "burgers": burgers,
        "ks": kuramoto_sivashinsky,
        "allen_cahn": allen_cahn,
        "helmholtz": helmholtz,
        "ns_psi": navier_stokes_psi,
        "ns_uvp": navier_stokes_uvp,
    }
    return table[name](**kw)
