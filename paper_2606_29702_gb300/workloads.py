"""Seeded synthetic workloads: collocation points, network shapes, parameters.

This module holds no arithmetic of the method.  It only draws random inputs
(uniform collocation points, Xavier-normal weights) and names the residual
family and its coefficients, so that the CUDA path and the FP64 oracle can be
fed identical inputs.  It imports neither.

The five workloads stand in for the paper's collocation sets (Sec. 3.1.1 uses
10000 / 10000 / 4096 PDE points and 6x64 tanh networks; no public dataset is
involved in the residual loss):

* ``burgers_2x20x4``: viscous Burgers, nu = 0.01/pi, 2->20x4->1, N = 1000
  uniform on [-1,1]x[0,1], float64.
* ``ks_2x64x5``: Kuramoto-Sivashinsky with unit coefficients, 2->64x5->1,
  N = 65536 uniform on [0,2pi]x[0,1], float32.
* ``ns_psi_3x128x6``: stream-function Navier-Stokes, nu = 0.01, 3->128x6->2,
  N = 262144 uniform on [0,1]^3, bf16 operands.
* ``ensemble_64``: 32 Burgers (nu log-uniform in [1e-3,1e-1]) and 32
  Allen-Cahn instances, widths {32,64,128}, 3..8 hidden layers,
  N_i uniform in [2048, 65536], bf16 operands.
* ``helmholtz_3x256x8``: 3-D Helmholtz, k = 4 pi, 3->256x8->1, N = 1048576
  uniform on [-1,1]^3, bf16 operands, Adam lr 1e-3.
* ``ns_uvp_2x64x6``: steady Navier-Stokes in primitive variables (u, v, p),
  Re = 100 (Eq. 16), 2->64x6->3 as in Sec. 3.1.1, N = 10000 PDE points
  uniform on the unit square, float32.

and the two composite losses of Sec. 3.1.1 (all points batched), see
``loss_workload``:

* ``burgers_loss_2x64x6``: Burgers on [0,1]^2, nu = 0.01, 1000 periodic
  boundary pairs ((0, t), (1, t)), 101 initial-condition points with
  u0(x) = -sin(2 pi x), 10000 PDE points; 2->64x6->1.
* ``cavity_loss_2x64x6``: the lid-driven cavity at Re = 100, 10000 PDE points,
  1499 no-slip wall points (x = 0, x = 1 or y = 0; u = v = 0) and 499 lid
  points (y = 1; u = 1, v = 0); 2->64x6->3.
"""

import math

import numpy as np

WORKLOADS = {
    "burgers_2x20x4": dict(family="burgers", coefs=dict(nu=0.01 / math.pi), widths=[2] + [20] * 4 + [1],
                           N=1000, domain=[(-1.0, 1.0), (0.0, 1.0)], precision="fp64", seed_pts=0, seed_par=1),
    "ks_2x64x5": dict(family="ks", coefs=dict(c1=1.0, c2=1.0, c4=1.0), widths=[2] + [64] * 5 + [1],
                      N=65536, domain=[(0.0, 2.0 * math.pi), (0.0, 1.0)], precision="fp32", seed_pts=0, seed_par=1),
    "ns_psi_3x128x6": dict(family="ns_psi", coefs=dict(nu=0.01), widths=[3] + [128] * 6 + [2],
                           N=262144, domain=[(0.0, 1.0)] * 3, precision="bf16", seed_pts=0, seed_par=1),
    "helmholtz_3x256x8": dict(family="helmholtz", coefs=dict(k=4.0 * math.pi), widths=[3] + [256] * 8 + [1],
                              N=1048576, domain=[(-1.0, 1.0)] * 3, precision="bf16", seed_pts=0, seed_par=1),
    "ns_uvp_2x64x6": dict(family="ns_uvp", coefs=dict(Re=100.0), widths=[2] + [64] * 6 + [3],
                          N=10000, domain=[(0.0, 1.0)] * 2, precision="fp32", seed_pts=0, seed_par=1),
}


def points(domain, N, seed):
    """N points uniform on the box ``domain`` = [(lo, hi), ...]; float64 [N, d]."""
    rng = np.random.default_rng(seed)
    lo = np.array([a for a, _ in domain], dtype=np.float64)
    hi = np.array([b for _, b in domain], dtype=np.float64)
    return lo + (hi - lo) * rng.random((N, len(domain)))


def xavier_layers(widths, seed, bias_std=0.0):
    """Xavier-normal weights, std = sqrt(2 / (fan_in + fan_out)); biases N(0, bias_std^2).

    Returns a list of (W [out, in], b [out]) float64 arrays.
    """
    rng = np.random.default_rng(seed)
    layers = []
    for fi, fo in zip(widths[:-1], widths[1:]):
        W = rng.standard_normal((fo, fi)) * math.sqrt(2.0 / (fi + fo))
        b = rng.standard_normal(fo) * bias_std if bias_std > 0 else np.zeros(fo)
        layers.append((W, b))
    return layers


def pack(layers):
    """(W, b) list -> flat vector: per layer W row-major then b (the ABI packing)."""
    return np.concatenate([np.concatenate([np.asarray(W).ravel(), np.asarray(b).ravel()]) for W, b in layers])


def unpack(flat, widths):
    flat = np.asarray(flat).ravel()
    out, off = [], 0
    for fi, fo in zip(widths[:-1], widths[1:]):
        W = flat[off:off + fo * fi].reshape(fo, fi)
        off += fo * fi
        out.append((W, flat[off:off + fo]))
        off += fo
    assert off == flat.size
    return out


def n_params(widths):
    return sum(fo * fi + fo for fi, fo in zip(widths[:-1], widths[1:]))


def workload(name, N=None, bias_std=0.0):
    """(spec dict, X [N, d] float64, layers) for a named workload."""
    spec = dict(WORKLOADS[name])
    n = spec["N"] if N is None else N
    X = points(spec["domain"], n, spec["seed_pts"])
    layers = xavier_layers(spec["widths"], spec["seed_par"], bias_std)
    return spec, X, layers


def ensemble(n_burgers=32, n_ac=32, widths=(32, 64, 128), depth=(3, 8), n_range=(2048, 65536), base_seed=100):
    """Instance list of the batched-ensemble workload.

    Instance i draws everything from seed base_seed + i: its width (uniform
    over ``widths``), its number of hidden layers (uniform in ``depth``), its
    point count (uniform in ``n_range``), its Burgers viscosity (log-uniform in
    [1e-3, 1e-1]), its points and its parameters.
    """
    out = []
    for i in range(n_burgers + n_ac):
        rng = np.random.default_rng(base_seed + i)
        w = int(rng.choice(widths))
        D = int(rng.integers(depth[0], depth[1] + 1))
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        if i < n_burgers:
            fam, coefs = "burgers", dict(nu=float(10.0 ** rng.uniform(-3.0, -1.0)))
        else:
            fam, coefs = "allen_cahn", dict(eps=1e-4, k=5.0)
        wid = [2] + [w] * D + [1]
        X = points([(-1.0, 1.0), (0.0, 1.0)], N, int(rng.integers(1 << 30)))
        layers = xavier_layers(wid, int(rng.integers(1 << 30)))
        out.append(dict(family=fam, coefs=coefs, widths=wid, N=N, X=X, layers=layers))
    return out


LOSS_WORKLOADS = {
    "burgers_loss_2x64x6": dict(kind="burgers", coefs=dict(nu=0.01), widths=[2] + [64] * 6 + [1],
                                counts=dict(bc_pairs=1000, ic=101, pde=10000), precision="fp32", seed_pts=0,
                                seed_par=1),
    "cavity_loss_2x64x6": dict(kind="cavity", coefs=dict(Re=100.0), widths=[2] + [64] * 6 + [3],
                               counts=dict(pde=10000, wall=1499, lid=499), precision="fp32", seed_pts=0, seed_par=1),
}


def loss_points(kind, counts, seed):
    """Concatenated points of a composite loss, in term order, with the
    per-term point counts and the per-point prescribed values (the source
    rows: the initial condition, the wall and lid velocities).

    Returns (X [N, 2], term counts, source [N, n_src] or None)."""
    rng = np.random.default_rng(seed)
    if kind == "burgers":
        nb, ni, npde = counts["bc_pairs"], counts["ic"], counts["pde"]
        t = rng.random(nb)
        bc = np.empty((2 * nb, 2))
        bc[0::2, 0], bc[1::2, 0] = 0.0, 1.0
        bc[0::2, 1] = bc[1::2, 1] = t
        xi = rng.random(ni)
        ic = np.column_stack([xi, np.zeros(ni)])
        pde = rng.random((npde, 2))
        X = np.concatenate([bc, ic, pde])
        src = np.zeros((X.shape[0], 2))  # [N][n_res]: the periodic term has two components
        src[2 * nb:2 * nb + ni, 0] = -np.sin(2.0 * math.pi * xi)
        return X, [2 * nb, ni, npde], src
    npde, nw, nl = counts["pde"], counts["wall"], counts["lid"]
    pde = rng.random((npde, 2))
    s = rng.random(nw)
    side = rng.integers(0, 3, nw)
    wall = np.column_stack([np.where(side == 0, 0.0, np.where(side == 1, 1.0, s)),
                            np.where(side == 2, 0.0, s)])
    lid = np.column_stack([rng.random(nl), np.ones(nl)])
    X = np.concatenate([pde, wall, lid])
    src = np.zeros((X.shape[0], 3))
    src[npde + nw:, 0] = 1.0
    return X, [npde, nw, nl], src


def loss_workload(name, scale=1.0):
    """(spec dict, X, term counts, source, layers) of a composite-loss
    workload; ``scale`` multiplies every point count (pairs stay pairs)."""
    spec = dict(LOSS_WORKLOADS[name])
    counts = {k: max(1, int(round(v * scale))) for k, v in spec["counts"].items()}
    X, cnt, src = loss_points(spec["kind"], counts, spec["seed_pts"])
    layers = xavier_layers(spec["widths"], spec["seed_par"])
    return spec, X, cnt, src, layers
