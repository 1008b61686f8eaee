"""Composite PINN losses with all-points batching (Sec. 3.1.1) on the GPU,
through the C ABI, against the composite-loss oracle (oracle/losses.py).

The two losses of the paper's experiments: Burgers with periodic boundary
pairs for u and u_x, an initial-condition term and the PDE residual; the
lid-driven cavity with the residuals of Eq. 16 and the wall and lid velocity
terms.  All points are concatenated in term order and evaluated once; each
term's residual is compared at its own points, the second points of pairs
must read zero, and the loss and gradient are compared as a whole.

Bounds (relative L2 of residuals / gradient, relative loss): FP64 1e-12 /
1e-10, FP32 the stated 1e-5, BF16 about twice the error measured on a GB300.
"""
import numpy as np
import pytest

from _common import rel_l2
from paper_2606_29702_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = {"burgers": dict(w_ic=3.0, w_bc=0.5, w_pde=1.0), "cavity": dict(w_wall=2.0, w_lid=0.5, w_pde=1.0)}
TOL = {"fp64": (1e-12, 1e-10), "fp32": (1e-5, 1e-5)}
TOL_BF16 = {"burgers_loss_2x64x6": (2.1e-2, 2.6e-2), "cavity_loss_2x64x6": (2.1e-2, 1.3e-2)}
CASES = [("burgers_loss_2x64x6", "fp64", 0.02), ("burgers_loss_2x64x6", "fp32", 0.1),
         ("burgers_loss_2x64x6", "bf16", 0.1), ("cavity_loss_2x64x6", "fp64", 0.02),
         ("cavity_loss_2x64x6", "fp32", 0.1), ("cavity_loss_2x64x6", "bf16", 0.1)]


def _terms(kind, coefs):
    from oracle import losses as Lo
    from paper_2606_29702_gb300 import specs
    if kind == "burgers":
        return (specs.burgers_loss_terms(coefs["nu"], **W[kind]), Lo.burgers_terms(coefs["nu"], **W[kind]))
    return specs.cavity_loss_terms(coefs["Re"], **W[kind]), Lo.cavity_terms(coefs["Re"], **W[kind])


def _oracle_sources(kind, X, counts, src):
    lo = np.cumsum([0] + counts)
    if kind == "burgers":
        return [None, src[lo[1]:lo[2], 0], None]
    return [None, src[lo[1]:lo[2], :2], src[lo[2]:lo[3], :2]]


def _setup(name, scale, bias_std=0.1):
    spec, X, counts, src, _ = wl.loss_workload(name, scale)
    layers = wl.xavier_layers(spec["widths"], spec["seed_par"] + 7, bias_std)
    return spec, X, counts, src, layers


@pytest.mark.parametrize("name,prec,scale", CASES, ids=["%s-%s" % (c[0], c[1]) for c in CASES])
def test_composite_loss_matches_oracle(name, prec, scale):
    from oracle import losses as Lo
    from paper_2606_29702_gb300 import jet
    spec, X, counts, src, layers = _setup(name, scale)
    lib_terms, or_terms = _terms(spec["kind"], spec["coefs"])
    L, res, grads = Lo.loss_and_grad(or_terms, counts, layers, X, _oracle_sources(spec["kind"], X, counts, src))
    g_ref = wl.pack(grads)
    plan = jet.LossPlan(lib_terms, spec["widths"], prec)
    plan.set_term_points(counts)
    dt = plan.dtype
    p = torch.tensor(wl.pack(layers), dtype=dt, device="cuda")
    x = torch.tensor(X, dtype=dt, device="cuda")
    s = torch.tensor(src, dtype=dt, device="cuda")
    r, loss = plan.forward(p, x, s)
    g, loss_b, r_b = plan.backward(p, x, s, want_r=True)
    torch.cuda.synchronize()
    r = r.cpu().double().numpy()
    tr, tg = TOL_BF16[name] if prec == "bf16" else TOL[prec]
    lo = np.cumsum([0] + counts)
    errs = []
    for k, (t, ref) in enumerate(zip(or_terms, res)):
        rows = r[lo[k]:lo[k + 1]]
        if t.paired:
            assert np.all(rows[1::2] == 0.0)  # second points of pairs
            rows = rows[0::2]
        assert np.all(rows[:, t.n_res:] == 0.0)
        errs.append(rel_l2(rows[:, :t.n_res], ref))
    eg = rel_l2(g.cpu().numpy(), g_ref)
    el = abs(float(loss) - L) / abs(L)
    print("LOSS %s %s: term residuals %s gradient %.3e loss %.3e (class %s)"
          % (name, prec, " ".join("%.2e" % e for e in errs), eg, el, plan.info()["class_name"]))
    assert max(errs) <= tr and eg <= tg and el <= 2 * tr
    assert torch.equal(torch.tensor(r), r_b.cpu().double()) and float(loss_b) == float(loss)


def test_composite_loss_in_a_batch_equals_solo():
    """Two composite-loss plans and a single-residual plan of the same channel
    set in one batched launch."""
    from paper_2606_29702_gb300 import jet, specs
    plans, ps, xs, ss = [], [], [], []
    for name, scale in (("burgers_loss_2x64x6", 0.05), ("burgers_loss_2x64x6", 0.13)):
        spec, X, counts, src, layers = _setup(name, scale)
        lib_terms, _ = _terms(spec["kind"], spec["coefs"])
        plan = jet.LossPlan(lib_terms, spec["widths"], "bf16")
        plan.set_term_points(counts)
        plans.append(plan)
        ps.append(torch.tensor(wl.pack(layers), dtype=torch.float32, device="cuda"))
        xs.append(torch.tensor(X, dtype=torch.float32, device="cuda"))
        ss.append(torch.tensor(src, dtype=torch.float32, device="cuda"))
    widths = [2, 64, 64, 64, 1]
    plans.append(jet.Plan(specs.burgers(0.01), widths, "bf16"))
    ps.append(torch.tensor(wl.pack(wl.xavier_layers(widths, 9, 0.1)), dtype=torch.float32, device="cuda"))
    xs.append(torch.tensor(wl.points([(0, 1), (0, 1)], 700, 9), dtype=torch.float32, device="cuda"))
    ss.append(None)
    solo = [pl.backward(p, x, s) for pl, p, x, s in zip(plans, ps, xs, ss)]
    grads, losses = jet.Batch(plans).backward(ps, xs, sources=ss)
    torch.cuda.synchronize()
    for i in range(3):
        assert rel_l2(grads[i].cpu().numpy(), solo[i][0].cpu().numpy()) < 1e-6
        assert abs(float(losses[i]) - float(solo[i][1])) <= 1e-12 * abs(float(solo[i][1]))


def test_composite_loss_call_checks():
    from paper_2606_29702_gb300 import jet
    spec, X, counts, src, layers = _setup("burgers_loss_2x64x6", 0.01)
    lib_terms, _ = _terms(spec["kind"], spec["coefs"])
    plan = jet.LossPlan(lib_terms, spec["widths"], "fp32")
    p = torch.tensor(wl.pack(layers), dtype=torch.float32, device="cuda")
    x = torch.tensor(X, dtype=torch.float32, device="cuda")
    s = torch.tensor(src, dtype=torch.float32, device="cuda")
    with pytest.raises(jet.JetError, match="set_term_points"):
        plan.forward(p, x, s)  # counts not given yet
    with pytest.raises(jet.JetError, match="even"):
        plan.set_term_points([counts[0] - 1, counts[1] + 1, counts[2]])  # a pair split
    plan.set_term_points([counts[0], counts[1], counts[2] - 1])
    with pytest.raises(jet.JetError, match="differs"):
        plan.forward(p, x, s)
    reordered = [lib_terms[1], lib_terms[0], lib_terms[2]]  # the paired term after an odd block
    plan2 = jet.LossPlan(reordered, spec["widths"], "fp32")
    with pytest.raises(jet.JetError, match="even"):
        plan2.set_term_points([counts[1], counts[0], counts[2]])
