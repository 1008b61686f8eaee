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
    from paper_2606_29702_gb300 import jet
    insts, plans, ps, xs = _ensemble(2, 2, (500, 3000), 21, prec)
    b = jet.Batch(plans)
    p_e = [p.clone() for p in ps]
    m_e = [torch.zeros_like(p) for p in ps]
    v_e = [torch.zeros_like(p) for p in ps]
    p_g = [p.clone() for p in ps]
    m_g = [torch.zeros_like(p) for p in ps]
    v_g = [torch.zeros_like(p) for p in ps]
    loss_e = torch.empty(len(plans), dtype=torch.float64, device="cuda")
    loss_g = torch.empty(len(plans), dtype=torch.float64, device="cuda")
    lr = float(np.float32(1e-3))
    # eager: three steps
    for step in (1, 2, 3):
        b.train_step(p_e, m_e, v_e, step, lr, xs, loss=loss_e)
    # graph: warm up once eagerly on a side stream, capture step 2, replay twice
    b.train_step(p_g, m_g, v_g, 1, lr, xs, loss=loss_g)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.train_step(p_g, m_g, v_g, 2, lr, xs, loss=loss_g)
    torch.cuda.synchronize()
    g.replay()  # step 2 (capture does not execute)
    torch.cuda.synchronize()
    step2 = [p.clone() for p in p_g]
    g.replay()  # replays the same step index: Adam bias correction of step 2 again
    torch.cuda.synchronize()
    # reference for "step 2 applied twice" from the eager state after step 2
    p_r = [p.clone() for p in ps]
    m_r = [torch.zeros_like(p) for p in ps]
    v_r = [torch.zeros_like(p) for p in ps]
    loss_r = torch.empty_like(loss_e)
    for step in (1, 2, 2):
        b.train_step(p_r, m_r, v_r, step, lr, xs, loss=loss_r)
    torch.cuda.synchronize()
    for i in range(len(plans)):
        assert torch.equal(p_g[i], p_r[i])
        assert not torch.equal(step2[i], p_g[i])
    assert torch.equal(loss_g, loss_r)


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
