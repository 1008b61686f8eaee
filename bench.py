"""Benchmark: residual + parameter-gradient collocation points/s on one GB300.

One step = one full pass of the hot path over one batch of collocation points:
jet forward (all channels, all layers), residual, loss, residual adjoint,
reverse sweep to the parameter gradient, FP64 reduction and the Adam update
(jet_train_step).

Headline (default): 3-D Helmholtz, 3->256x8->1 tanh MLP, N = 1048576 points
uniform on [-1,1]^3, BF16 tensor-core form, Adam lr 1e-3 -- the largest
single-GPU configuration.  Beside it, in the same run and under named keys
("workloads"): the other schedule of the same workload, its plain FP32 form,
the stream-function Navier-Stokes 3->128x6->2 (BF16, BF16X3, FP32), the
Kuramoto-Sivashinsky 2->64x5->1 (FP32, BF16, BF16X3), the FP64 Burgers
2->20x4->1 and the 64-instance batched ensemble in BF16 and in plain FP32.

``--workload ensemble_64`` makes the batched form the headline: 64
independent PINNs (32 Burgers, 32 Allen-Cahn; widths 32/64/128, 3-8 hidden
layers, N_i in [2048, 65536]) trained together by one persistent launch per
step, captured in a CUDA graph whose Adam step counter lives on the device.

``--train K`` runs K Adam steps of the headline workload after 20 warm-up
steps (Sec. 3.1.1: 1000 steps, lr 1e-3) and reports the time per step and the
loss history.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica of the workload (the
points are independent; no collective on the data path): weak scaling.
"""

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "residual+param-grad collocation pts/s on 1 GB300; TC roofline %; rel err vs FP64"
UNIT = "points/s"
L2_BYTES = 129 * 1024 * 1024
STORE_BUDGET = 96 << 30  # HBM the tensor-core forms may use for the weight-gradient store


HEADLINE = "helmholtz_3x256x8"
# the named workloads timed beside the headline: (workload, form, schedule)
SIDE = [("helmholtz_3x256x8", "bf16", "store"), ("helmholtz_3x256x8", "bf16", "tile"),
        ("helmholtz_3x256x8", "fp32", "tile"),
        ("ns_psi_3x128x6", "bf16", "tile"), ("ns_psi_3x128x6", "bf16x3", "tile"), ("ns_psi_3x128x6", "fp32", "tile"),
        ("ks_2x64x5", "fp32", "tile"), ("ks_2x64x5", "bf16", "tile"), ("ks_2x64x5", "bf16x3", "tile"),
        ("burgers_2x20x4", "fp64", "tile"),
        ("burgers_loss_2x64x6", "fp32", "tile"), ("burgers_loss_2x64x6", "bf16", "tile"),
        ("cavity_loss_2x64x6", "fp32", "tile"), ("cavity_loss_2x64x6", "bf16", "tile"),
        ("ensemble_64", "bf16", "tile"), ("ensemble_64", "fp32", "tile")]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=HEADLINE)
    ap.add_argument("--form", default=None, help="precision form of the headline (default: the workload's)")
    ap.add_argument("--schedule", default=None, choices=["tile", "store"],
                    help="weight-gradient schedule of a tensor-core headline (default: the workload's)")
    ap.add_argument("--no-forms", action="store_true", help="time the headline only")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="0 skips the oracle leg")
    ap.add_argument("--n", type=int, default=None, help="override the workload's point count (profiling)")
    ap.add_argument("--train", type=int, default=0, help="K > 0: a K-step Adam training run of the headline")
    ap.add_argument("--history", default=None, help="--train: write the loss history (JSON) here")
    return ap.parse_args()


def dist_init():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, ws, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(ms_local, n_local, ws):
    """(max step time over ranks, whole-job points/s): every rank runs an
    independent replica of n_local points, timed by the slowest rank."""
    ms = max_over_ranks(ms_local, ws)
    return ms, ws * n_local / (ms * 1e-3)


def flops_per_point(widths, C):
    """Algorithmic jet-GEMM flops per point of one step: forward, data gradient
    and weight gradient of every hidden-to-hidden layer, 2 C w_in w_out each."""
    f = sum(2.0 * C * widths[l - 1] * widths[l] for l in range(2, len(widths) - 1))
    return 3.0 * f


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


def fp32_alu_peak_tflops(sm_mhz=2070.0, sms=152):
    """FP32 FMA peak: 152 SMs x 128 FP32 lanes x 2 flop x SM clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


# DRAM bytes (read + write) of one launch of the dominant kernel, from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum) on the same workload, form
# and schedule; (workload, form, schedule) -> (bytes per launch, hash of the
# kernel sources the counters were taken on).  A different hash (the kernels
# changed since) gives null.  Entries taken on a smaller N than the workload's
# are scaled by the point count where the traffic is per tile (stated in the
# profile summaries).
TRAFFIC = {
    # N = 65536 capture of both kernels (fused kernel + weight-gradient GEMM): the store's bytes x16; the GEMM's
    # per-item FP32 partials (one per CTA and layer, the same at any N) once
    ("helmholtz_3x256x8", "bf16", "store"): ((647555328 + 3771561472 + 3759028736) * 16 + 239769856, "69ceaa525bc23bd5"),
    ("ns_psi_3x128x6", "bf16", "tile"): (21527552 + 2450227712, "69ceaa525bc23bd5"),
    ("ks_2x64x5", "bf16", "tile"): (853504 + 1003008, "69ceaa525bc23bd5"),
    ("ks_2x64x5", "fp32", "tile"): (14223360 + 813413888, "69ceaa525bc23bd5"),
    # the batched fused kernel of one ensemble step (the step is one graph replay)
    ("ensemble_64", "bf16", "tile"): (846524416 + 2861984000, "69ceaa525bc23bd5"),
}


def kernel_source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2606_29702_gb300", "csrc")
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h", ".py")) and name != "jet_closures_gen.h":
            with open(os.path.join(d, name), "rb") as f:
                h.update(name.encode())
                h.update(f.read())
    return h.hexdigest()[:16]


def traffic_for(workload, form, schedule="tile"):
    e = TRAFFIC.get((workload, form, schedule))
    return e[0] if e is not None and e[1] == kernel_source_hash() else None


def roofline(form, flops, kernel_ms, peaks, peak_kind, traffic=None):
    """Roofline of the dominant kernel: algorithmic jet-GEMM flops / its event time."""
    achieved = flops / (kernel_ms * 1e-3) / 1e12
    if form in ("fp32", "fp64"):
        peak = fp32_alu_peak_tflops(peaks.get("sm_max_mhz", 2070.0)) if form == "fp32" else \
            fp64_alu_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "fused SIMT jet kernel (%s)" % form,
                "peak_kind": "derived: 152 SM x %s lanes x 2 flop x max clock" % ("128 FP32" if form == "fp32"
                                                                                 else "2 FP64")}
    peak = peaks["bf16_tflops"] * (0.5 if form == "tf32" else 1.0)
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": "tcgen05 fused jet kernel (%s)" % form,
            "peak_kind": "%s bf16_tflops (burst)" % peak_kind}


def fp64_alu_peak_tflops(sm_mhz=2070.0, sms=152):
    """FP64 FMA peak: 152 SMs x 2 FP64 FMA per clock x 2 flop x SM clock, the
    nominal 1.25 TFLOP/s of a GB300."""
    return sms * 2 * 2 * sm_mhz * 1e6 / 1e12


# ------------------------------------------------------------------ reference
def run_reference(args, rank, ws):
    """The oracle (FP64 NumPy) as it stands on the host cores, on a bounded
    sample of the workload per step (for the ensemble: 32 points of every
    instance per step)."""
    if rank != 0:
        return
    import oracle
    from oracle import residuals as R
    from paper_2606_29702_gb300 import workloads as wl
    jobs = []  # (residual family, widths, points, packed params, source)
    if args.workload == "ensemble_64":
        for ins in wl.ensemble():
            jobs.append((R.by_name(ins["family"], **ins["coefs"]), ins["widths"], ins["X"][:32],
                         wl.pack(ins["layers"]), None))
        widths, sample = "32/64/128, 3-8 hidden layers", "32 points of each of the 64 instances per step"
    else:
        spec = wl.WORKLOADS[args.workload]
        X = wl.points(spec["domain"], 256, spec["seed_pts"])
        src = R.helmholtz_source(X, spec["coefs"]["k"])[:, None] if spec["family"] == "helmholtz" else None
        jobs.append((R.by_name(spec["family"], **spec["coefs"]), spec["widths"], X,
                     wl.pack(wl.xavier_layers(spec["widths"], spec["seed_par"])), src))
        widths, sample = spec["widths"], "256 of the workload's points per step"
    S = sum(j[2].shape[0] for j in jobs)
    state = [(j[3], np.zeros_like(j[3]), np.zeros_like(j[3])) for j in jobs]

    def step(k):
        for i, (fam, wid, X, _, src) in enumerate(jobs):
            theta, m, v = state[i]
            _, _, g = oracle.loss_and_grad(fam, wl.unpack(theta, wid), X, source=src)
            state[i] = oracle.adam_step(theta, m, v, wl.pack(g), k + 1)

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(args.warmup + k)
    dt = (time.perf_counter() - t0) / args.steps
    cores = _blas_threads()
    val = S / dt
    out = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": args.workload, "points_per_step": S, "widths": widths,
                      "note": "FP64 oracle (hyper-dual jets + reverse tape), bounded sample per step"},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": "%s, %d steps" % (sample, args.steps)},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


def cpu_baseline(spec, seconds, forms=()):
    """Oracle points/s on the host cores over a bounded sample (~`seconds` s),
    and the relative error against it of every GPU form on the same sample."""
    import oracle
    from oracle import residuals as R
    from paper_2606_29702_gb300 import workloads as wl
    S = 256
    X = wl.points(spec["domain"], S, spec["seed_pts"] + 7)
    layers = wl.xavier_layers(spec["widths"], spec["seed_par"])
    fam = R.by_name(spec["family"], **spec["coefs"])
    src = R.helmholtz_source(X, spec["coefs"]["k"])[:, None] if spec["family"] == "helmholtz" else None
    L_ref, r_ref, g_ref = oracle.loss_and_grad(fam, layers, X, source=src)
    g_ref = wl.pack(g_ref)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        oracle.loss_and_grad(fam, layers, X, source=src)
        n += 1
    dt = time.perf_counter() - t0
    errs = {}
    for f in forms:
        try:
            r, g = gpu_sample(spec, f, X, layers, src)
            errs[f] = {"residual_rel_l2": float(np.linalg.norm(r - r_ref) / np.linalg.norm(r_ref)),
                       "gradient_rel_l2": float(np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref))}
        except Exception as e:  # a form this build does not provide
            errs[f] = {"unavailable": str(e).splitlines()[0][:120]}
    return {"value": n * S / max(dt, 1e-9), "unit": UNIT, "cores": _blas_threads(), "kind": "oracle",
            "sample": "%d runs of residual+gradient on %d points of the workload (%.1f s)" % (n, S, dt)}, errs


def gpu_sample(spec, form, X, layers, src):
    """Residual and gradient of one GPU form on the sample points (float64 numpy)."""
    import torch
    from paper_2606_29702_gb300 import jet, specs
    from paper_2606_29702_gb300 import workloads as wl
    plan = jet.Plan(specs.by_name(spec["family"], **spec["coefs"]), spec["widths"], form)
    dt = plan.dtype
    p = torch.tensor(wl.pack(layers), dtype=dt, device="cuda")
    x = torch.tensor(X, dtype=dt, device="cuda")
    s = None if src is None else torch.tensor(src, dtype=dt, device="cuda")
    g, _, r = plan.backward(p, x, s, want_r=True)
    torch.cuda.synchronize()
    out = r.cpu().double().numpy(), g.cpu().double().numpy()
    plan.close()
    return out


# ------------------------------------------------------------------ ours
DTYPES = {"fp32": "f32", "fp64": "f64", "bf16": "bf16", "tf32": "tf32", "bf16x3": "bf16x3"}


def default_schedule(spec, form):
    """Weight-gradient schedule of a tensor-core form: the store (layer inputs
    and adjoints of every tile in HBM, one weight-gradient GEMM per layer) for
    width-256 layers, where it measured 3x faster; per-tile flushes otherwise."""
    return "store" if form in ("bf16", "bf16x3") and max(spec["widths"][1:-1]) >= 256 else "tile"


def launches_per_step(form, schedule, batched=False, dev_counter=False):
    """Kernels of ours one train step launches (memsets excluded)."""
    if form in ("fp32", "fp64"):
        n = 3  # weight transposition (one per member when batched), fused SIMT kernel, reduce + Adam
    else:
        n = 3 if schedule == "tile" else 5  # weight prep, fused tcgen05 kernel, [wgrad GEMM, wgrad sum], reduce
    return n + (1 if dev_counter else 0)


def make_plan(spec, form, schedule):
    from paper_2606_29702_gb300 import jet, specs
    sp = specs.by_name(spec["family"], **spec["coefs"])
    kw = dict(store=True, mem_budget=STORE_BUDGET) if schedule == "store" else {}
    return sp, jet.Plan(sp, spec["widths"], form, **kw)


def time_form(spec, form, X_host, steps, warmup, flush, want_kernel=False, e2e=False, schedule="tile"):
    """Time `steps` train steps of one precision form and schedule; returns a dict."""
    import torch
    from paper_2606_29702_gb300 import specs
    from paper_2606_29702_gb300 import workloads as wl
    sp, plan = make_plan(spec, form, schedule)
    dt = plan.dtype
    dev = torch.device("cuda")
    layers = wl.xavier_layers(spec["widths"], spec["seed_par"])
    p = torch.tensor(wl.pack(layers), dtype=dt, device=dev)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    x = torch.tensor(X_host, dtype=dt, device=dev)
    src = None
    if sp.has_source:
        src = torch.tensor(specs.helmholtz_source(X_host, spec["coefs"]["k"]), dtype=dt, device=dev)
    loss = torch.empty((), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    step = 1
    for _ in range(warmup):
        plan.train_step(p, m, v, step, 1e-3, x, src, loss)
        step += 1
    torch.cuda.synchronize()
    if want_kernel:
        plan.profile(True)
        plan.profile_read()
    evs = []
    for _ in range(steps):
        flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.train_step(p, m, v, step, 1e-3, x, src, loss)
        b.record(stream)
        evs.append((a, b))
        step += 1
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    out = {"ms_per_step": ms, "value": X_host.shape[0] / (ms * 1e-3), "info": plan.info(), "schedule": schedule,
           "loss": float(loss)}
    if want_kernel:
        n, kms = plan.profile_read()
        plan.profile(False)
        out["kernel_ms"] = kms / max(n, 1)
        out["kernel_launches"] = n
    if e2e:
        # public API end to end: pinned host X -> device, step, loss -> host
        xh = torch.tensor(X_host, dtype=dt).pin_memory()
        lh = torch.empty((), dtype=torch.float64).pin_memory()
        xd = torch.empty_like(x)
        evs = []
        for _ in range(steps):
            flush()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            xd.copy_(xh, non_blocking=True)
            plan.train_step(p, m, v, step, 1e-3, xd, src, loss)
            lh.copy_(loss, non_blocking=True)
            b.record(stream)
            evs.append((a, b))
            step += 1
        torch.cuda.synchronize()
        ems = sum(a.elapsed_time(b) for a, b in evs) / steps
        out["e2e"] = {"value": X_host.shape[0] / (ems * 1e-3), "unit": UNIT,
                      "h2d_bytes_per_step": int(xh.numel() * xh.element_size()),
                      "d2h_bytes_per_step": int(lh.numel() * lh.element_size())}
    plan.close()
    return out


def time_ensemble(form, steps, warmup, rank=0, e2e=True):
    """Batched ensemble: one graph-captured jet_batch_train_step_dev per step
    (the Adam step counter lives on the device, so every replay is the next
    step).  Returns a dict with the per-step time and the points of a replica."""
    import torch
    from paper_2606_29702_gb300 import autotune, jet, specs
    from paper_2606_29702_gb300 import workloads as wl
    insts = wl.ensemble(base_seed=100 + 1000 * rank)
    dev = torch.device("cuda")
    ps = [torch.tensor(wl.pack(i["layers"]), dtype=torch.float32, device=dev) for i in insts]
    ms_ = [torch.zeros_like(p) for p in ps]
    vs = [torch.zeros_like(p) for p in ps]
    xh = [torch.tensor(i["X"], dtype=torch.float32).pin_memory() for i in insts]
    xs = [x.to(dev) for x in xh]
    # tiles autotuned on the batch itself (CTA shape and tile scale timed as
    # whole batched launches, cached per batch shape), outside the timed region
    members = [(specs.by_name(i["family"], **i["coefs"]), i["widths"], p) for i, p in zip(insts, ps)]
    plans = autotune.batch_plans(members, form, xs)
    tune = autotune.load_cache().get(autotune.batch_key(members, form), {})
    tiles = [p.info()["tile_points"] for p in plans]
    n_pts = sum(i["N"] for i in insts)
    loss = torch.empty(len(insts), dtype=torch.float64, device=dev)
    ctr = torch.zeros(1, dtype=torch.int64, device=dev)
    batch = jet.Batch(plans)
    flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    W = max(warmup, 3)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for k in range(W):
            batch.train_step_dev(ps, ms_, vs, ctr, 1e-3, xs, loss=loss, stream=s)
    torch.cuda.synchronize()
    # one step captured as a CUDA graph (descriptor uploads, weight preparation,
    # the persistent batched kernel, the batched FP64 reduce + Adam and the
    # step-counter advance)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batch.train_step_dev(ps, ms_, vs, ctr, 1e-3, xs, loss=loss, stream=s)
    g.replay()  # the first launch of a graph also uploads it: untimed
    torch.cuda.synchronize()
    evs = []
    for _ in range(steps):
        flush_buf.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    out = {"ms_per_step": ms, "value": n_pts / (ms * 1e-3), "n_pts": n_pts, "insts": insts, "tune": tune,
           "tiles": tiles, "adam_steps_taken": int(ctr.item()), "loss_mean": float(loss.mean())}
    if e2e:
        # end to end: pinned host points in, losses out, every step
        lh = torch.empty(len(insts), dtype=torch.float64).pin_memory()
        evs = []
        for _ in range(steps):
            flush_buf.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            for xd, xp in zip(xs, xh):
                xd.copy_(xp, non_blocking=True)
            g.replay()
            lh.copy_(loss, non_blocking=True)
            b.record()
            evs.append((a, b))
        torch.cuda.synchronize()
        out["e2e_ms"] = sum(a.elapsed_time(b) for a, b in evs) / steps
        out["h2d"] = int(sum(x.numel() * x.element_size() for x in xh))
        out["d2h"] = int(lh.numel() * lh.element_size())
    batch.close()
    for p in plans:
        p.close()
    return out


def ensemble_flops(insts):
    return sum(i["N"] * flops_per_point(i["widths"], 4) for i in insts)


def run_ensemble(args, rank, ws, local):
    """The batched ensemble as the headline."""
    form = args.form or "bf16"
    W = max(args.warmup, 3)
    clocks = Clocks(local)
    barrier(ws)
    clocks.start()
    res = time_ensemble(form, args.steps, W, rank)
    barrier(ws)
    clk = clocks.stop()
    insts = res["insts"]
    ms, value = aggregate(res["ms_per_step"], res["n_pts"], ws)
    e2e_ms = max_over_ranks(res["e2e_ms"], ws)
    peaks, peak_kind = measured_peaks()
    roof = roofline(form, ensemble_flops(insts), res["ms_per_step"], peaks, peak_kind,
                    traffic_for("ensemble_64", form))
    roof["kernel"] = "batched step (graph replay: weight preparation, persistent fused kernel, reduce + Adam)"
    tune = res["tune"]
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": W,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": DTYPES[form], "data": "synthetic",
           "config": {"workload": "ensemble_64", "instances": len(insts), "points_per_replica": res["n_pts"],
                      "widths": sorted(set(i["widths"][1] for i in insts)),
                      "depths": [min(len(i["widths"]) - 2 for i in insts), max(len(i["widths"]) - 2 for i in insts)],
                      "form": form,
                      "tiles": "autotuned on the batch: %s CTA(s)/SM, %g x each shape's default tile (%s points); "
                               "options timed (ms): %s" % (tune.get("ctas"), tune.get("scale", 1.0),
                                                          ",".join(str(t) for t in sorted(set(res["tiles"]))),
                                                          tune.get("ms")),
                      "l2": "flushed between steps (2x L2 write, outside the per-step events)",
                      "step": "jet_batch_train_step_dev of all instances, one CUDA graph replay"},
           "e2e": {"value": ws * res["n_pts"] / (e2e_ms * 1e-3), "unit": UNIT,
                   "h2d_bytes_per_step": res["h2d"], "d2h_bytes_per_step": res["d2h"]},
           "gpu_launches": launches_per_step(form, "tile", True, True) * args.steps, "roofline": roof,
           "clocks": clk, "cpu_baseline": None}
    if rank == 0:
        print(json.dumps(out))


def time_loss_form(name, form, steps, warmup, flush):
    """Train steps of a composite-loss workload (Sec. 3.1.1: IC, BC and PDE
    terms over their own points, all points batched into one evaluation)."""
    import torch
    from paper_2606_29702_gb300 import jet, specs
    from paper_2606_29702_gb300 import workloads as wl
    spec, X, counts, src, layers = wl.loss_workload(name)
    terms = specs.burgers_loss_terms(**spec["coefs"]) if spec["kind"] == "burgers" else \
        specs.cavity_loss_terms(**spec["coefs"])
    plan = jet.LossPlan(terms, spec["widths"], form)
    plan.set_term_points(counts)
    dev = torch.device("cuda")
    p = torch.tensor(wl.pack(layers), dtype=plan.dtype, device=dev)
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    x = torch.tensor(X, dtype=plan.dtype, device=dev)
    s = torch.tensor(src, dtype=plan.dtype, device=dev)
    loss = torch.empty((), dtype=torch.float64, device=dev)
    for k in range(warmup):
        plan.train_step(p, m, v, k + 1, 1e-3, x, s, loss)
    torch.cuda.synchronize()
    plan.profile(True)
    plan.profile_read()
    evs = []
    for k in range(steps):
        flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        plan.train_step(p, m, v, warmup + k + 1, 1e-3, x, s, loss)
        b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    n, kms = plan.profile_read()
    info = plan.info()
    plan.close()
    return {"ms_per_step": ms, "value": X.shape[0] / (ms * 1e-3), "kernel_ms": kms / max(n, 1), "info": info,
            "points": X.shape[0], "counts": counts, "widths": spec["widths"]}


def side_entry(name, form, schedule, steps, flush, peaks, peak_kind):
    """One named workload timed beside the headline (rank 0, one replica)."""
    from paper_2606_29702_gb300 import workloads as wl
    if name in wl.LOSS_WORKLOADS:
        r = time_loss_form(name, form, steps, 3, flush)
        fpp = flops_per_point(r["widths"], r["info"]["n_channels"])
        return {"value": r["value"], "ms_per_step": r["ms_per_step"], "kernel_ms": r["kernel_ms"],
                "points": r["points"], "term_points": r["counts"], "form": form,
                "tile_points": r["info"]["tile_points"], "channels": r["info"]["n_channels"],
                "step": "jet_train_step on the composite loss (all points batched)",
                "roofline": roofline(form, fpp * r["points"], r["kernel_ms"], peaks, peak_kind, None)}
    if name == "ensemble_64":
        r = time_ensemble(form, steps, 3, e2e=False)
        return {"value": r["value"], "ms_per_step": r["ms_per_step"], "points": r["n_pts"], "form": form,
                "step": "one CUDA graph replay of jet_batch_train_step_dev",
                "roofline": dict(roofline(form, ensemble_flops(r["insts"]), r["ms_per_step"], peaks, peak_kind,
                                          traffic_for(name, form)),
                                 kernel="batched step (graph replay)")}
    spec = dict(wl.WORKLOADS[name])
    X = wl.points(spec["domain"], spec["N"], spec["seed_pts"])
    r = time_form(spec, form, X, steps, 3, flush, want_kernel=True, schedule=schedule)
    fpp = flops_per_point(spec["widths"], r["info"]["n_channels"])
    return {"value": r["value"], "ms_per_step": r["ms_per_step"], "kernel_ms": r["kernel_ms"], "points": spec["N"],
            "form": form, "schedule": schedule, "tile_points": r["info"]["tile_points"],
            "grid_ctas": r["info"]["grid_ctas"], "channels": r["info"]["n_channels"],
            "roofline": roofline(form, fpp * spec["N"], r["kernel_ms"], peaks, peak_kind,
                                 traffic_for(name, form, schedule))}


def run_ours(args, rank, ws, local):
    import torch
    if args.workload == "ensemble_64":
        return run_ensemble(args, rank, ws, local)
    from paper_2606_29702_gb300 import workloads as wl
    spec = dict(wl.WORKLOADS[args.workload])
    if args.n:
        spec["N"] = args.n
    form = args.form or spec["precision"]
    schedule = args.schedule or default_schedule(spec, form)
    X = wl.points(spec["domain"], spec["N"], spec["seed_pts"] + rank)
    flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def flush():
        flush_buf.fill_(1.0)

    if args.train:
        return run_train(args, spec, form, schedule, X, rank, ws, local)
    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    res = time_form(spec, form, X, args.steps, max(args.warmup, 3), flush, want_kernel=True, e2e=True,
                    schedule=schedule)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    ms, value = aggregate(res["ms_per_step"], spec["N"], ws)
    C = res["info"]["n_channels"]
    fpp = flops_per_point(spec["widths"], C)
    peaks, peak_kind = measured_peaks()
    roof = roofline(form, fpp * spec["N"], res["kernel_ms"], peaks, peak_kind,
                    traffic_for(args.workload, form, schedule))
    if schedule == "store":
        roof["kernel"] += " + store weight-gradient GEMM"
    side = {}
    if not args.no_forms and rank == 0:
        for name, f, sc in SIDE:
            if (name, f, sc) == (args.workload, form, schedule):
                continue
            key = "%s/%s/%s" % (name, f, sc)
            try:
                side[key] = side_entry(name, f, sc, max(3, args.steps // 2), flush, peaks, peak_kind)
            except Exception as e:  # a form this build does not provide
                side[key] = {"unavailable": str(e).splitlines()[0][:160]}
            torch.cuda.empty_cache()
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": DTYPES[form], "data": "synthetic",
           "config": {"workload": args.workload, "N": spec["N"], "widths": spec["widths"], "form": form,
                      "schedule": schedule, "channels": C, "tile_points": res["info"]["tile_points"],
                      "l2": "flushed between steps (2x L2 write, outside the per-step events)",
                      "step": "jet_train_step: forward jets + residual + loss + reverse sweep + FP64 reduce + Adam"},
           "e2e": res["e2e"], "gpu_launches": launches_per_step(form, schedule) * args.steps, "roofline": roof,
           "clocks": clk, "workloads": side}
    if rank == 0:
        if ws == 1 and args.cpu_seconds > 0:
            forms = [form] + sorted({f for n, f, _ in SIDE if n == args.workload and f != form})
            out["cpu_baseline"], out["rel_err_vs_fp64"] = cpu_baseline(spec, args.cpu_seconds, forms)
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out))


def run_train(args, spec, form, schedule, X, rank, ws, local):
    """K Adam steps (lr 1e-3) after 20 warm-up steps on a fresh initialisation,
    with the loss of every step kept on the device (Sec. 3.1.1 protocol: 1000
    steps, 20 warm-up steps, CUDA events around the steps)."""
    import torch
    from paper_2606_29702_gb300 import specs
    from paper_2606_29702_gb300 import workloads as wl
    sp, plan = make_plan(spec, form, schedule)
    dt = plan.dtype
    dev = torch.device("cuda")
    p0 = torch.tensor(wl.pack(wl.xavier_layers(spec["widths"], spec["seed_par"])), dtype=dt, device=dev)
    x = torch.tensor(X, dtype=dt, device=dev)
    src = torch.tensor(specs.helmholtz_source(X, spec["coefs"]["k"]), dtype=dt, device=dev) if sp.has_source \
        else None
    K, W = args.train, 20
    # warm-up on a scratch copy, so that the timed run starts at step 1
    pw, mw, vw = p0.clone(), torch.zeros_like(p0), torch.zeros_like(p0)
    cw = torch.zeros(1, dtype=torch.int64, device=dev)
    for _ in range(W):
        plan.train_step_dev(pw, mw, vw, cw, 1e-3, x, src)
    p, m, v = p0.clone(), torch.zeros_like(p0), torch.zeros_like(p0)
    ctr = torch.zeros(1, dtype=torch.int64, device=dev)
    hist = torch.empty(K, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for k in range(K):
        plan.train_step_dev(p, m, v, ctr, 1e-3, x, src, loss=hist[k])
    b.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = a.elapsed_time(b) / K
    h = hist.cpu().numpy()
    out = {"metric": METRIC, "value": spec["N"] / (ms * 1e-3), "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
           "ms_per_step": ms, "total_s": ms * K / 1e3, "dtype": DTYPES[form], "data": "synthetic",
           "config": {"workload": args.workload, "N": spec["N"], "widths": spec["widths"], "form": form,
                      "schedule": schedule, "lr": 1e-3, "adam_steps": int(ctr.item()),
                      "step": "jet_train_step_dev, one call per step, no L2 flush between steps"},
           "loss_first": float(h[0]), "loss_last": float(h[-1]),
           "loss_every_50": [float(h[i]) for i in range(0, K, 50)] + [float(h[-1])], "clocks": clk}
    if args.history:
        with open(args.history, "w") as f:
            json.dump({"loss": h.tolist(), **{k: out[k] for k in ("config", "ms_per_step")}}, f)
    if rank == 0:
        print(json.dumps(out))
    plan.close()


def main():
    args = parse()
    rank, ws, local = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, ws)
    else:
        run_ours(args, rank, ws, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
