"""Plain FP64 PINN residual, loss, gradient and Adam step.

Test infrastructure only (see ``oracle/__init__.py``).

Passages followed:
* Eq. 1 (Sec. 2.2): z^l = W^l a^{l-1} + b^l, a^l = phi(z^l), phi = tanh for the
  hidden layers.  The output layer is linear (standard PINN reading; the paper
  applies phi at every layer of Eq. 1 but its networks map to physical fields).
* Sec. 2.2: r_theta(x) = N(u_theta, d_i u_theta, d_ij u_theta, ...), the
  coordinate derivatives of the network output.  They are computed here by
  nested hyper-dual numbers, one run per multi-index, NOT by the layerwise
  rules of Eq. 2-3.
* Sec. 3.1.1: the parameter gradient is the reverse-mode derivative of the
  scalar loss; here L = sum_c (1/N) sum_n r_{c,n}^2 (mean-squared residual of
  each residual component, summed over components), differentiated by the
  generic tape of ``tape.py``.
* Sec. 3.1.1: full-batch Adam with learning rate 1e-3; beta1 = 0.9,
  beta2 = 0.999, eps = 1e-8 with bias correction (Kingma & Ba 2015; the paper
  gives only the learning rate).

Parameter packing (shared convention with the library ABI, pure layout): for
each layer l = 1..L in order, W^l row-major [out, in] followed by b^l [out].

Parity: every function is pinned by tests/test_oracle_pins.py.
"""

import numpy as np

from . import hyperdual as hd
from .tape import Var, backward


def unpack_params(packed, widths):
    """Packed vector -> list of (W [out,in], b [out]) float64 arrays."""
    packed = np.asarray(packed, dtype=np.float64).ravel()
    out, off = [], 0
    for fi, fo in zip(widths[:-1], widths[1:]):
        W = packed[off:off + fo * fi].reshape(fo, fi)
        off += fo * fi
        b = packed[off:off + fo]
        off += fo
        out.append((W, b))
    if off != packed.size:
        raise ValueError("packed parameter vector has %d entries, widths need %d" % (packed.size, off))
    return out


def pack_params(layers):
    return np.concatenate([np.concatenate([np.asarray(W).ravel(), np.asarray(b).ravel()]) for W, b in layers])


def _mlp(layers, h, act):
    """Eq. 1 applied layer by layer; linear output layer."""
    L = len(layers)
    for l, (W, b) in enumerate(layers):
        Wt = W.T
        h = h @ Wt + b
        if l < L - 1:
            h = act(h)
    return h


def network_jets(layers, X, channels, act=hd.tanh):
    """d^alpha u(x_n) for every multi-index alpha in ``channels``.

    layers: list of (W, b) (numpy arrays or tape Vars); X: [N, d] points.
    Returns {alpha: [N, n_out]} (numpy arrays or tape Vars).
    """
    out = {}
    for alpha in channels:
        alpha = tuple(int(k) for k in alpha)
        dirs = hd.dirs_of(alpha)
        x = hd.seed_input(X, dirs)
        y = _mlp(layers, x, act)
        out[alpha] = hd.top_coefficient(y, len(dirs))
    return out


def _values(x):
    return x.value if isinstance(x, Var) else np.asarray(x, dtype=np.float64)


def residual(family, layers, X, act=hd.tanh, source=None):
    """r [N, n_res] for a residual family from ``oracle.residuals``."""
    X = np.asarray(X, dtype=np.float64)
    jets = network_jets(layers, X, family.needed, act)
    comps = family.components(jets, X, source)
    return np.stack([np.broadcast_to(_values(c), (X.shape[0],)) for c in comps], axis=1)


def loss_value(family, layers, X, act=hd.tanh, source=None):
    r = residual(family, layers, X, act, source)
    return float((r * r).sum() / r.shape[0])


def loss_and_grad(family, layers, X, act=hd.tanh, source=None):
    """(L, r [N, n_res], grads) with grads a list of (dL/dW, dL/db) per layer."""
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    vlayers = [(Var(np.array(W, dtype=np.float64)), Var(np.array(b, dtype=np.float64))) for W, b in layers]
    jets = network_jets(vlayers, X, family.needed, act)
    comps = family.components(jets, X, source)
    loss = None
    for c in comps:
        if not isinstance(c, Var):
            raise TypeError("a residual component does not depend on the parameters")
        term = (c * c).sum() * (1.0 / N)
        loss = term if loss is None else loss + term
    r = np.stack([c.value for c in comps], axis=1)
    backward(loss)
    grads = []
    for W, b in vlayers:
        gW = W.grad if W.grad is not None else np.zeros_like(W.value)
        gb = b.grad if b.grad is not None else np.zeros_like(b.value)
        grads.append((gW, gb))
    return float(loss.value), r, grads


def adam_step(theta, m, v, g, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One bias-corrected Adam update (Kingma & Ba 2015, Algorithm 1); step >= 1."""
    theta = np.asarray(theta, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
