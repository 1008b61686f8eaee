"""Batched ensembles on the tensor cores (one persistent launch over a work
list of instance chunks), CUDA-graph capture of the batched train step, and
the tile autotuner, all through the C ABI."""
import numpy as np
import pytest

from _common import rel_l2
from paper_2606_29702_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ensemble(n_b, n_ac, n_range, seed, prec="bf16"):
    from paper_2606_29702_gb300 import jet, specs
    insts = wl.ensemble(n_burgers=n_b, n_ac=n_ac, widths=(32, 64, 128), depth=(3, 8), n_range=n_range,
                        base_seed=seed)
    plans, ps, xs = [], [], []
    for ins in insts:
        plans.append(jet.Plan(specs.by_name(ins["family"], **ins["coefs"]), ins["widths"], prec))
        ps.append(torch.tensor(wl.pack(ins["layers"]), dtype=torch.float32, device="cuda"))
        xs.append(torch.tensor(ins["X"], dtype=torch.float32, device="cuda"))
    return insts, plans, ps, xs


def test_tc_batch_matches_solo_and_oracle():
    import oracle
    from oracle import residuals as R
    from paper_2606_29702_gb300 import jet
    insts, plans, ps, xs = _ensemble(3, 3, (100, 1500), 11)
    solo = [p.backward(a, x) for p, a, x in zip(plans, ps, xs)]
    b = jet.Batch(plans)
    grads, losses = b.backward(ps, xs)
    torch.cuda.synchronize()
    # batch and solo runs chunk the tiles differently; a chunk's weight
    # gradients add up in FP32 (about T * 2^-24 relative for T tiles), the
    # chunks in FP64
    for i, ins in enumerate(insts):
        assert rel_l2(grads[i].cpu().numpy(), solo[i][0].cpu().numpy()) < 1e-6
        assert abs(float(losses[i]) - float(solo[i][1])) <= 1e-12 * abs(float(solo[i][1]))
        L, _, g_ref = oracle.loss_and_grad(R.by_name(ins["family"], **ins["coefs"]), ins["layers"], ins["X"])
        assert rel_l2(grads[i].cpu().numpy(), wl.pack(g_ref)) < 3e-2
        assert abs(float(losses[i]) - L) / L < 3e-2


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_batch_train_step_graph_replay_equals_eager(prec):
    """A captured batched train step with the Adam step counter in device
    memory: three replays of one graph equal three eager steps 1, 2, 3
    (bitwise), and the counter reads 3 afterwards."""
    from paper_2606_29702_gb300 import jet
    insts, plans, ps, xs = _ensemble(2, 2, (500, 3000), 21, prec)
    b = jet.Batch(plans)
    lr = float(np.float32(1e-3))

    def state():
        return [p.clone() for p in ps], [torch.zeros_like(p) for p in ps], [torch.zeros_like(p) for p in ps]

    p_e, m_e, v_e = state()
    loss_e = torch.empty(len(plans), dtype=torch.float64, device="cuda")
    for step in (1, 2, 3):
        b.train_step(p_e, m_e, v_e, step, lr, xs, loss=loss_e)
    # the device counter, eagerly: same steps, same bits
    p_d, m_d, v_d = state()
    ctr_d = torch.zeros(1, dtype=torch.int64, device="cuda")
    loss_d = torch.empty_like(loss_e)
    for _ in range(3):
        b.train_step_dev(p_d, m_d, v_d, ctr_d, lr, xs, loss=loss_d)
    # captured once (a warm-up call on a scratch copy first), replayed three times
    p_g, m_g, v_g = state()
    ctr = torch.zeros(1, dtype=torch.int64, device="cuda")
    loss_g = torch.empty_like(loss_e)
    p_w, m_w, v_w = state()
    b.train_step_dev(p_w, m_w, v_w, torch.zeros(1, dtype=torch.int64, device="cuda"), lr, xs)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.train_step_dev(p_g, m_g, v_g, ctr, lr, xs, loss=loss_g, stream=s)
    torch.cuda.synchronize()
    assert int(ctr.item()) == 0  # capture does not execute
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert int(ctr.item()) == 3 and int(ctr_d.item()) == 3
    for i in range(len(plans)):
        assert torch.equal(p_d[i], p_e[i]) and torch.equal(m_d[i], m_e[i]) and torch.equal(v_d[i], v_e[i])
        assert torch.equal(p_g[i], p_e[i]) and torch.equal(m_g[i], m_e[i]) and torch.equal(v_g[i], v_e[i])
    assert torch.equal(loss_g, loss_e) and torch.equal(loss_d, loss_e)


@pytest.mark.parametrize("prec", ["bf16", "fp32", "fp64"])
def test_plan_train_step_graph_replay_equals_eager(prec):
    """jet_train_step_dev on one plan: three replays of a captured step equal
    jet_train_step with steps 1, 2, 3 (bitwise)."""
    import math
    from paper_2606_29702_gb300 import jet, specs
    widths = [2, 64, 64, 64, 1]
    plan = jet.Plan(specs.burgers(0.01 / math.pi), widths, prec)
    dt = plan.dtype
    layers = wl.xavier_layers(widths, 5, bias_std=0.1)
    x = torch.tensor(wl.points([(-1, 1), (0, 1)], 1500, 6), dtype=dt, device="cuda")
    p0 = torch.tensor(wl.pack(layers), dtype=dt, device="cuda")
    lr = float(np.float32(1e-3))
    p_e, m_e, v_e = p0.clone(), torch.zeros_like(p0), torch.zeros_like(p0)
    for step in (1, 2, 3):
        loss_e = plan.train_step(p_e, m_e, v_e, step, lr, x)
    p_w, m_w, v_w = p0.clone(), torch.zeros_like(p0), torch.zeros_like(p0)
    plan.train_step_dev(p_w, m_w, v_w, torch.zeros(1, dtype=torch.int64, device="cuda"), lr, x)
    torch.cuda.synchronize()
    p_g, m_g, v_g = p0.clone(), torch.zeros_like(p0), torch.zeros_like(p0)
    ctr = torch.zeros(1, dtype=torch.int64, device="cuda")
    loss_g = torch.empty((), dtype=torch.float64, device="cuda")
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.train_step_dev(p_g, m_g, v_g, ctr, lr, x, loss=loss_g, stream=s)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert int(ctr.item()) == 3
    assert torch.equal(p_g, p_e) and torch.equal(m_g, m_e) and torch.equal(v_g, v_e)
    assert torch.equal(loss_g, loss_e)


def test_full_ensemble_one_launch():
    """The 64-instance ensemble (32 Burgers, 32 Allen-Cahn; widths 32/64/128,
    3-8 hidden layers, N_i in [2048, 65536]) in one batched call; a sample of
    instances against their solo runs."""
    from paper_2606_29702_gb300 import jet
    insts, plans, ps, xs = _ensemble(32, 32, (2048, 65536), 100)
    b = jet.Batch(plans)
    grads, losses = b.backward(ps, xs)
    torch.cuda.synchronize()
    for i in (0, 17, 40, 63):
        g, l, _ = plans[i].backward(ps[i], xs[i])
        torch.cuda.synchronize()
        assert rel_l2(grads[i].cpu().numpy(), g.cpu().numpy()) < 1e-6  # FP32 chunk sums, as above
    assert torch.isfinite(losses).all()


def test_autotune_on_gpu(tmp_path):
    from paper_2606_29702_gb300 import autotune, jet, specs
    sp = specs.ks()
    widths = [2, 64, 64, 64, 1]
    X = wl.points([(0, 6.28), (0, 1)], 4096, 3)
    layers = wl.xavier_layers(widths, 4)
    p = torch.tensor(wl.pack(layers), dtype=torch.float32, device="cuda")
    x = torch.tensor(X, dtype=torch.float32, device="cuda")
    path = str(tmp_path / "tune.json")
    best, res = autotune.tune(sp, widths, "bf16", p, x, candidates=(8, 16, 32, 40), path=path)
    assert best in res and len(res) >= 2
    tuned = autotune.plan(sp, widths, "bf16", path=path)
    assert tuned.info()["tile_points"] == best
    g1, l1, _ = tuned.backward(p, x)
    g0, l0, _ = jet.Plan(sp, widths, "bf16").backward(p, x)
    torch.cuda.synchronize()
    assert rel_l2(g1.cpu().numpy(), g0.cpu().numpy()) < 1e-5


def test_batch_autotune_on_gpu(tmp_path):
    """tune_batch times whole batched launches under each option that fits;
    batch_plans builds the chosen plans from the cache, and their batch gives
    the solo gradients (up to FP32 chunk-sum rounding)."""
    from paper_2606_29702_gb300 import autotune, jet, specs
    insts, plans0, ps, xs = _ensemble(2, 2, (1500, 4000), 31)
    members = [(specs.by_name(i["family"], **i["coefs"]), i["widths"], p) for i, p in zip(insts, ps)]
    path = str(tmp_path / "tune.json")
    best, res = autotune.tune_batch(members, "bf16", xs, reps=1, path=path)
    assert best in res and (1, 1.0) in res
    plans = autotune.batch_plans(members, "bf16", xs, path=path)
    grads, losses = jet.Batch(plans).backward(ps, xs)
    torch.cuda.synchronize()
    for i in range(len(insts)):
        g, l, _ = plans0[i].backward(ps[i], xs[i])
        torch.cuda.synchronize()
        assert rel_l2(grads[i].cpu().numpy(), g.cpu().numpy()) < 1e-3
        assert abs(float(losses[i]) - float(l)) <= 1e-5 * abs(float(l))


def test_simt_batch_with_fp32_accumulator():
    """FP32 SIMT members wide enough that their FP64 slices leave L2 add their
    weight gradients in per-CTA FP32 accumulators; in a batch, every chunk item
    zeroes and flushes its own, and the gradients match the solo runs and the
    oracle."""
    import oracle
    from oracle import residuals as R
    from paper_2606_29702_gb300 import jet, specs
    sp = specs.ns_psi(0.01)
    widths = [3, 128, 128, 128, 128, 2]
    plans, ps, xs, refs = [], [], [], []
    for k, n in enumerate((97, 180)):
        layers = wl.xavier_layers(widths, 40 + k, bias_std=0.1)
        X = wl.points([(0, 1)] * 3, n, 50 + k)
        plans.append(jet.Plan(sp, widths, "fp32"))
        ps.append(torch.tensor(wl.pack(layers), dtype=torch.float32, device="cuda"))
        xs.append(torch.tensor(X, dtype=torch.float32, device="cuda"))
        refs.append(oracle.loss_and_grad(R.by_name("ns_psi", nu=0.01), layers, X))
    assert all(p.info()["wgrad_chunk_fp32"] == 1 for p in plans)
    grads, losses = jet.Batch(plans).backward(ps, xs)
    torch.cuda.synchronize()
    for i in range(2):
        g, l, _ = plans[i].backward(ps[i], xs[i])
        torch.cuda.synchronize()
        assert rel_l2(grads[i].cpu().numpy(), g.cpu().numpy()) < 1e-6
        L, _, g_ref = refs[i]
        assert rel_l2(grads[i].cpu().double().numpy(), wl.pack(g_ref)) < 1e-5
        assert abs(float(losses[i]) - L) <= 1e-5 * abs(L)
