"""Residual specifications of the PDE families as monomial tables for libjet.

A residual component is sum_m coef_m prod_j d^{alpha_j} u_{o_j} minus an
optional per-point source (Sec. 2.2: r_theta = N(u, d_i u, d_ij u, ...)).
Multi-indices are tuples of derivative orders per input coordinate.

Families (coordinates in input order):
* burgers(nu), inputs (x, t): u_t + u u_x - nu u_xx (Sec. 3.1.1).
* ks(c1, c2, c4), inputs (x, t): u_t + c1 u u_x + c2 u_xx + c4 u_xxxx
  (Sec. 3.1.1).
* allen_cahn(eps, k), inputs (x, t): u_t - eps u_xx + k u^3 - k u.
* helmholtz(k), inputs (x, y, z): u_xx + u_yy + u_zz + k^2 u - f, f passed as
  the source column.
* ns_psi(nu), inputs (x, y, t), outputs (psi, p), u = psi_y, v = -psi_x:
  the momentum residuals of Eq. 16 with the time derivative,
  r_u = psi_yt + psi_y psi_xy - psi_x psi_yy + p_x - nu (psi_xxy + psi_yyy),
  r_v = -psi_xt - psi_y psi_xx + psi_x psi_xy + p_y + nu (psi_xxx + psi_xyy).
* ns_uvp(Re), inputs (x, y), outputs (u, v, p): the steady incompressible
  Navier-Stokes residuals of Eq. 16 in primitive variables,
  r_c = u_x + v_y,
  r_u = u u_x + v u_y + p_x - (u_xx + u_yy) / Re,
  r_v = u v_x + v v_y + p_y - (v_xx + v_yy) / Re
  (closure {0, x, y, xx, yy}: no mixed channel).
"""

import math


class Spec:
    def __init__(self, name, d_in, n_out, components, has_source=False):
        self.name = name
        self.d_in = d_in
        self.n_out = n_out
        self.components = components  # [[(coef, [(o, alpha), ...]), ...], ...]
        self.has_source = has_source

    @property
    def n_res(self):
        return len(self.components)

    def needed(self):
        s = {tuple([0] * self.d_in)}
        for comp in self.components:
            for _, facs in comp:
                for _, al in facs:
                    s.add(tuple(al))
        return sorted(s)

    def closure(self):
        out = set()
        for al in self.needed():
            stack = [tuple(al)]
            while stack:
                a = stack.pop()
                if a in out:
                    continue
                out.add(a)
                for i, k in enumerate(a):
                    if k > 0:
                        b = list(a)
                        b[i] -= 1
                        stack.append(tuple(b))
        return sorted(out, key=lambda a: (sum(a), a))


def burgers(nu):
    X, T, XX, U = (1, 0), (0, 1), (2, 0), (0, 0)
    return Spec("burgers", 2, 1, [[(1.0, [(0, T)]), (1.0, [(0, U), (0, X)]), (-nu, [(0, XX)])]])


def ks(c1=1.0, c2=1.0, c4=1.0):
    return Spec("ks", 2, 1, [[(1.0, [(0, (0, 1))]), (c1, [(0, (0, 0)), (0, (1, 0))]),
                              (c2, [(0, (2, 0))]), (c4, [(0, (4, 0))])]])


def allen_cahn(eps=1e-4, k=5.0):
    U = (0, 0)
    return Spec("allen_cahn", 2, 1, [[(1.0, [(0, (0, 1))]), (-eps, [(0, (2, 0))]),
                                      (k, [(0, U), (0, U), (0, U)]), (-k, [(0, U)])]])


def helmholtz(k=4.0 * math.pi):
    return Spec("helmholtz", 3, 1, [[(1.0, [(0, (2, 0, 0))]), (1.0, [(0, (0, 2, 0))]), (1.0, [(0, (0, 0, 2))]),
                                     (k * k, [(0, (0, 0, 0))])]], has_source=True)


def ns_psi(nu=0.01):
    def a(x=0, y=0, t=0):
        return (x, y, t)
    ps, pr = 0, 1
    ru = [(1.0, [(ps, a(y=1, t=1))]), (1.0, [(ps, a(y=1)), (ps, a(x=1, y=1))]),
          (-1.0, [(ps, a(x=1)), (ps, a(y=2))]), (1.0, [(pr, a(x=1))]),
          (-nu, [(ps, a(x=2, y=1))]), (-nu, [(ps, a(y=3))])]
    rv = [(-1.0, [(ps, a(x=1, t=1))]), (-1.0, [(ps, a(y=1)), (ps, a(x=2))]),
          (1.0, [(ps, a(x=1)), (ps, a(x=1, y=1))]), (1.0, [(pr, a(y=1))]),
          (nu, [(ps, a(x=3))]), (nu, [(ps, a(x=1, y=2))])]
    return Spec("ns_psi", 3, 2, [ru, rv])


def ns_uvp(Re=100.0):
    U, X, Y, XX, YY = (0, 0), (1, 0), (0, 1), (2, 0), (0, 2)
    u, v, p = 0, 1, 2
    rc = [(1.0, [(u, X)]), (1.0, [(v, Y)])]
    ru = [(1.0, [(u, U), (u, X)]), (1.0, [(v, U), (u, Y)]), (1.0, [(p, X)]),
          (-1.0 / Re, [(u, XX)]), (-1.0 / Re, [(u, YY)])]
    rv = [(1.0, [(u, U), (v, X)]), (1.0, [(v, U), (v, Y)]), (1.0, [(p, Y)]),
          (-1.0 / Re, [(v, XX)]), (-1.0 / Re, [(v, YY)])]
    return Spec("ns_uvp", 2, 3, [rc, ru, rv])


# jet_chan.out flag of a factor read at the second point of a pair (JET_PAIR_SECOND)
PAIR_SECOND = 0x100


def burgers_loss_terms(nu=0.01, w_ic=1.0, w_bc=1.0, w_pde=1.0):
    """Composite Burgers loss of Sec. 3.1.1 as (spec, weight, paired) terms, in
    point order: periodic boundary pairs ((0, t), (1, t)) for u and u_x, the
    initial condition u(x, 0) - u0(x) (u0 per point as the source) and the
    PDE residual."""
    U, X = (0, 0), (1, 0)
    b = PAIR_SECOND
    bc = Spec("periodic_bc", 2, 1, [[(1.0, [(0, U)]), (-1.0, [(b, U)])], [(1.0, [(0, X)]), (-1.0, [(b, X)])]])
    ic = Spec("ic", 2, 1, [[(1.0, [(0, U)])]], has_source=True)
    return [(bc, w_bc, True), (ic, w_ic, False), (burgers(nu), w_pde, False)]


def cavity_loss_terms(Re=100.0, w_wall=1.0, w_lid=1.0, w_pde=1.0):
    """Composite lid-driven cavity loss of Sec. 3.1.1: the residuals of Eq. 16
    and the velocity conditions of the no-slip walls and of the lid, u - u_b
    and v - v_b with (u_b, v_b) per point as the source."""
    U = (0, 0)
    vel = [[(1.0, [(0, U)])], [(1.0, [(1, U)])]]
    return [(ns_uvp(Re), w_pde, False), (Spec("wall", 2, 3, vel, has_source=True), w_wall, False),
            (Spec("lid", 2, 3, vel, has_source=True), w_lid, False)]


FAMILIES = {"burgers": burgers, "ks": ks, "allen_cahn": allen_cahn, "helmholtz": helmholtz, "ns_psi": ns_psi,
            "ns_uvp": ns_uvp}
# representative coefficients of every family (the build derives each
# family's compiled channel set from its closure, which they do not change)
FAMILY_DEFAULTS = {"burgers": dict(nu=0.01), "ks": dict(), "allen_cahn": dict(), "helmholtz": dict(),
                   "ns_psi": dict(nu=0.01), "ns_uvp": dict(Re=100.0)}


def by_name(name, **coefs):
    return FAMILIES[name](**coefs)


def helmholtz_source(X, k=4.0 * math.pi):
    """Manufactured source f = (k^2 - 3 pi^2) sin(pi x) sin(pi y) sin(pi z) (numpy, float64)."""
    import numpy as np
    X = np.asarray(X, dtype=np.float64)
    pi = math.pi
    return ((k * k - 3 * pi * pi) * np.sin(pi * X[:, 0]) * np.sin(pi * X[:, 1]) * np.sin(pi * X[:, 2]))[:, None]
