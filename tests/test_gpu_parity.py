"""GPU parity of the SIMT forms (FP64, plain FP32) against the FP64 oracle.

Every call goes through the C ABI (ctypes binding).  Tolerances (relative L2
over points, and over the packed gradient):
  FP64: residual <= 1e-12, gradient <= 1e-10;
  FP32: residual <= 1e-5, gradient <= 1e-5 (the stated FP32 bound).
"""
import math

import numpy as np
import pytest

from _common import case, cosine, rel_l2, reference
from paper_2606_29702_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-12, 1e-10), "fp32": (1e-5, 1e-5)}


def _jet():
    from paper_2606_29702_gb300 import jet, specs
    return jet, specs


def _run(spec, X, layers, src, prec, plan=None):
    jet, specs = _jet()
    sp = specs.by_name(spec["family"], **spec["coefs"])
    plan = plan or jet.Plan(sp, spec["widths"], prec)
    dt = plan.dtype
    dev = torch.device("cuda")
    p = torch.tensor(wl.pack(layers), dtype=dt, device=dev)
    x = torch.tensor(X, dtype=dt, device=dev)
    s = None if src is None else torch.tensor(src, dtype=dt, device=dev)
    r, loss = plan.forward(p, x, s)
    g, loss_b, r_b = plan.backward(p, x, s, want_r=True)
    torch.cuda.synchronize()
    return (r.cpu().double().numpy(), float(loss), g.cpu().double().numpy(), float(loss_b),
            r_b.cpu().double().numpy(), plan)


CASES = [
    ("burgers_2x20x4", "fp64", 1000, None),
    ("burgers_2x20x4", "fp32", 1000, None),
    ("ks_2x64x5", "fp32", 300, None),
    ("ks_2x64x5", "fp64", 300, None),
    ("ns_psi_3x128x6", "fp32", 75, None),
    ("ns_psi_3x128x6", "fp64", 40, None),
    ("helmholtz_3x256x8", "fp32", 90, None),
    ("helmholtz_3x256x8", "fp64", 33, [3, 64, 64, 64, 1]),
    ("ns_uvp_2x64x6", "fp32", 500, None),
    ("ns_uvp_2x64x6", "fp64", 200, None),
]


@pytest.mark.parametrize("name,prec,N,widths", CASES, ids=["%s-%s-%d" % (c[0], c[1], c[2]) for c in CASES])
def test_simt_matches_oracle(name, prec, N, widths):
    spec, X, layers, src = case(name, N, widths=widths)
    L, r_ref, g_ref = reference(spec, X, layers)
    r, loss, g, loss_b, r_b, _ = _run(spec, X, layers, src, prec)
    tr, tg = TOL[prec]
    assert rel_l2(r, r_ref) <= tr, rel_l2(r, r_ref)
    assert rel_l2(g, g_ref) <= tg, rel_l2(g, g_ref)
    assert abs(loss - L) <= tr * abs(L) and abs(loss_b - L) <= tr * abs(L)
    assert cosine(g, g_ref) > 1 - 1e-9
    np.testing.assert_array_equal(r_b, r)


@pytest.mark.parametrize("name,N,chunk_fp32", [("ks_2x64x5", 999, 0), ("ns_psi_3x128x6", 301, 1)])
def test_simt_fp32_weight_gradient_paths(name, N, chunk_fp32):
    """FP32 plans whose per-chunk FP64 gradient slices fit in L2 add weight
    gradients into them per tile; wider ones accumulate a chunk's tiles in
    FP32 first.  Either way each sum has one owner thread and a fixed order:
    repeated calls are bitwise identical, and both match the oracle."""
    spec, X, layers, src = case(name, N)
    L, r_ref, g_ref = reference(spec, X, layers)
    r, loss, g, _, _, plan = _run(spec, X, layers, src, "fp32")
    assert plan.info()["wgrad_chunk_fp32"] == chunk_fp32
    assert rel_l2(g, g_ref) <= TOL["fp32"][1]
    for _ in range(2):
        _, _, g2, _, _, _ = _run(spec, X, layers, src, "fp32", plan=plan)
        np.testing.assert_array_equal(g2, g)


@pytest.mark.parametrize("N", [1, 2, 7, 47, 48, 49, 100])
def test_ragged_tails_fp64(N):
    spec, X, layers, src = case("burgers_2x20x4", N, seed_shift=N)
    L, r_ref, g_ref = reference(spec, X, layers)
    r, loss, g, _, _, _ = _run(spec, X, layers, src, "fp64")
    assert rel_l2(r, r_ref) <= 1e-12 and rel_l2(g, g_ref) <= 1e-10


def test_empty_input():
    jet, specs = _jet()
    spec, X, layers, _ = case("burgers_2x20x4", 4)
    plan = jet.Plan(specs.by_name("burgers", **spec["coefs"]), spec["widths"], "fp64")
    p = torch.tensor(wl.pack(layers), device="cuda")
    x = torch.empty((0, 2), dtype=torch.float64, device="cuda")
    r, loss = plan.forward(p, x)
    g, lb, _ = plan.backward(p, x)
    torch.cuda.synchronize()
    assert r.shape == (0, 1) and float(loss) == 0.0 and float(lb) == 0.0
    assert torch.count_nonzero(g).item() == 0


def test_full_size_ks_sampled_residuals_and_additivity():
    """KS 2->64x5->1 at N = 65536 in the launch the benchmark times: sampled
    residuals against the oracle point by point, and gradient additivity
    N * g(all) = N_a * g(first part) + N_b * g(rest) (any size)."""
    jet, specs = _jet()
    spec, X, layers, _ = case("ks_2x64x5", 65536, bias_std=0.0)
    plan = jet.Plan(specs.by_name("ks", **spec["coefs"]), spec["widths"], "fp32")
    p = torch.tensor(wl.pack(layers), dtype=torch.float32, device="cuda")
    x = torch.tensor(X, dtype=torch.float32, device="cuda")
    g, loss, r = plan.backward(p, x, want_r=True)
    idx = np.random.default_rng(0).choice(65536, 256, replace=False)
    import oracle
    from oracle import residuals as R
    Xs = x.cpu().double().numpy()[idx]
    r_ref = oracle.residual(R.by_name("ks", **spec["coefs"]), layers, Xs)
    assert rel_l2(r.cpu().double().numpy()[idx], r_ref) <= 1e-5
    na = 40000
    ga, _, _ = plan.backward(p, x[:na].contiguous())
    gb, _, _ = plan.backward(p, x[na:].contiguous())
    torch.cuda.synchronize()
    comb = (na * ga.double() + (65536 - na) * gb.double()) / 65536
    assert rel_l2(g.cpu().numpy(), comb.cpu().numpy()) <= 1e-5
    rr = r.cpu().double().numpy()
    assert abs(float(loss) - float((rr ** 2).mean())) <= 1e-5 * float(loss)


def test_store_equals_recompute():
    jet, specs = _jet()
    spec, X, layers, _ = case("ks_2x64x5", 500)
    sp = specs.by_name("ks", **spec["coefs"])
    plan_s = jet.Plan(sp, spec["widths"], "fp64", mem_budget=1 << 28, store=True)
    assert plan_s.info()["store_mode"] == 1
    plan_r = jet.Plan(sp, spec["widths"], "fp64")
    p = torch.tensor(wl.pack(layers), device="cuda")
    x = torch.tensor(X, device="cuda")
    plan_s.forward(p, x)
    g_s, l_s, _ = plan_s.backward(p, x)
    g_r, l_r, _ = plan_r.backward(p, x)
    torch.cuda.synchronize()
    assert torch.equal(g_s, g_r) and float(l_s) == float(l_r)


CLASS_SPECS = [
    ("d1", 1, [[(1.0, [(0, (4,))]), (1.0, [(0, (0,)), (0, (1,))])]]),
    ("d2o2", 2, [[(1.0, [(0, (1, 1))]), (0.5, [(0, (0, 2)), (0, (2, 0))])]]),
    ("d3o2", 3, [[(1.0, [(0, (1, 0, 1))]), (2.0, [(0, (0, 1, 1)), (0, (0, 0, 0))]), (-1.0, [(0, (0, 0, 2))])]]),
]


@pytest.mark.parametrize("name,d,comps", CLASS_SPECS, ids=[c[0] for c in CLASS_SPECS])
def test_generic_channel_sets_fp64(name, d, comps):
    import oracle
    from oracle import residuals as R
    jet, specs = _jet()
    sp = specs.Spec(name, d, 1, comps)
    widths = [d, 12, 16, 1]
    layers = wl.xavier_layers(widths, 3, bias_std=0.2)
    X = wl.points([(-1, 1)] * d, 61, 4)
    fam = R.monomial_family(d, 1, comps)
    L, r_ref, g_ref = oracle.loss_and_grad(fam, layers, X)
    plan = jet.Plan(sp, widths, "fp64")
    p = torch.tensor(wl.pack(layers), device="cuda")
    x = torch.tensor(X, device="cuda")
    r, loss = plan.forward(p, x)
    g, _, _ = plan.backward(p, x)
    torch.cuda.synchronize()
    assert rel_l2(r.cpu().numpy(), r_ref) <= 1e-12
    assert rel_l2(g.cpu().numpy(), wl.pack(g_ref)) <= 1e-10


@pytest.mark.parametrize("family", ["burgers", "ks", "ns_psi", "helmholtz"])
def test_activation_adjoint_inner_product(family):
    """Eq. 15: <J v, w> = <v, J^T w> for the activation-jet tangent J (FP64),
    and the tangent matches central differences of the composition."""
    jet, specs = _jet()
    coefs = {"burgers": dict(nu=0.01), "ks": {}, "ns_psi": dict(nu=0.01), "helmholtz": {}}[family]
    sp = specs.by_name(family, **coefs)
    plan = jet.Plan(sp, [sp.d_in, 8, sp.n_out], "fp64")
    C = plan.info()["n_channels"]
    g = np.random.default_rng(1)
    n = 1000
    z = torch.tensor(g.normal(size=(n, C)), device="cuda")
    v = torch.tensor(g.normal(size=(n, C)), device="cuda")
    w = torch.tensor(g.normal(size=(n, C)), device="cuda")
    Jv = plan.debug_activation(1, z, v)
    JTw = plan.debug_activation(2, z, w)
    lhs = (Jv * w).sum(1)
    rhs = (v * JTw).sum(1)
    # error relative to the size of the products being summed (cancellation-safe)
    scale = (Jv * w).abs().sum(1) + (v * JTw).abs().sum(1)
    err = ((lhs - rhs).abs() / scale).max().item()
    assert err < 1e-14, err
    h = 1e-6
    fd = (plan.debug_activation(0, z + h * v) - plan.debug_activation(0, z - h * v)) / (2 * h)
    assert rel_l2(fd.cpu().numpy(), Jv.cpu().numpy()) < 1e-8


def test_train_step_matches_oracle_adam():
    import oracle
    from oracle import residuals as R
    jet, specs = _jet()
    spec, X, layers, _ = case("burgers_2x20x4", 300)
    fam = R.by_name("burgers", **spec["coefs"])
    plan = jet.Plan(specs.by_name("burgers", **spec["coefs"]), spec["widths"], "fp64")
    theta = wl.pack(layers)
    p = torch.tensor(theta, device="cuda")
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    x = torch.tensor(X, device="cuda")
    th, mm, vv = theta.copy(), np.zeros_like(theta), np.zeros_like(theta)
    lr = float(np.float32(1e-3))  # the ABI passes the learning rate as a C float
    for step in range(1, 4):
        loss = plan.train_step(p, m, v, step, lr, x)
        L, _, gr = oracle.loss_and_grad(fam, wl.unpack(th, spec["widths"]), X)
        th, mm, vv = oracle.adam_step(th, mm, vv, wl.pack(gr), step, lr=lr)
        torch.cuda.synchronize()
        assert abs(float(loss) - L) <= 1e-12 * abs(L)
    assert rel_l2(p.cpu().numpy(), th) <= 1e-12
    assert rel_l2(m.cpu().numpy(), mm) <= 1e-10


def test_autograd_function_and_fd():
    """KS through torch.autograd.Function: FP32 gradient against the oracle and
    FP64 central differences of the loss along random directions."""
    jet, specs = _jet()
    spec, X, layers, _ = case("ks_2x64x5", 256)
    sp = specs.by_name("ks", **spec["coefs"])
    L, _, g_ref = reference(spec, X, layers)
    for prec in ("fp32", "fp64"):
        plan = jet.Plan(sp, spec["widths"], prec)
        p = torch.tensor(wl.pack(layers), dtype=plan.dtype, device="cuda", requires_grad=True)
        x = torch.tensor(X, dtype=plan.dtype, device="cuda")
        r, loss = jet.JetResidual.apply(p, x, plan, None)
        (3.0 * loss).backward()
        g = p.grad.detach().cpu().double().numpy() / 3.0
        assert rel_l2(g, g_ref) <= TOL[prec][1]
    plan64 = jet.Plan(sp, spec["widths"], "fp64")
    p64 = torch.tensor(wl.pack(layers), device="cuda")
    x64 = torch.tensor(X, device="cuda")
    rng = np.random.default_rng(3)
    for _ in range(3):
        d = rng.standard_normal(p64.numel())
        d = torch.tensor(d / np.linalg.norm(d), device="cuda")  # unit direction: truncation O(h^2) ~ 1e-8
        h = 1e-4
        lp = float(plan64.forward(p64 + h * d, x64, want_r=False)[1])
        lm = float(plan64.forward(p64 - h * d, x64, want_r=False)[1])
        fd = (lp - lm) / (2 * h)
        assert abs(fd - float(np.dot(g_ref, d.cpu().numpy()))) <= 1e-6 * abs(fd) + 1e-9


def test_batch_matches_solo_runs():
    jet, specs = _jet()
    insts = wl.ensemble(n_burgers=3, n_ac=3, widths=(32, 64, 128), depth=(3, 5), n_range=(100, 900), base_seed=7)
    plans, ps, xs, solo = [], [], [], []
    for ins in insts:
        sp = specs.by_name(ins["family"], **ins["coefs"])
        pl = jet.Plan(sp, ins["widths"], "fp32")
        p = torch.tensor(wl.pack(ins["layers"]), dtype=torch.float32, device="cuda")
        x = torch.tensor(ins["X"], dtype=torch.float32, device="cuda")
        plans.append(pl)
        ps.append(p)
        xs.append(x)
        g, loss, _ = pl.backward(p, x)
        solo.append((g, float(loss)))
    b = jet.Batch(plans)
    grads, losses = b.backward(ps, xs)
    torch.cuda.synchronize()
    import oracle
    from oracle import residuals as R
    for i, ins in enumerate(insts):
        L, _, g_ref = oracle.loss_and_grad(R.by_name(ins["family"], **ins["coefs"]), ins["layers"], ins["X"])
        assert rel_l2(grads[i].cpu().numpy(), wl.pack(g_ref)) <= 1e-5
        assert rel_l2(grads[i].cpu().numpy(), solo[i][0].cpu().numpy()) <= 1e-6
        assert abs(float(losses[i]) - L) <= 1e-5 * abs(L)


def test_ns_uvp_carries_exactly_its_closure():
    """Eq. 16 needs {0, x, y, xx, yy} for (u, v) and {0, x, y} for p: the plan
    carries the five-channel set built from the residual's spec, not a superset
    with the mixed xy channel."""
    jet, specs = _jet()
    for prec in ("fp32", "bf16"):
        plan = jet.Plan(specs.ns_uvp(100.0), [2, 64, 64, 3], prec)
        info = plan.info()
        assert info["class_name"] == "ns_uvp" and info["n_channels"] == 5
        plan.close()
