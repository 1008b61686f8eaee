"""jet_backward_params_noalloc against jet_backward_params (GPU).

The allocation-free entry point serves callers that cannot call cudaMalloc
(and so cannot create a plan): it keeps its working memory in a fixed 8 MiB
device array inside the library.  Its gradient and loss must equal those of
the plan-based entry point within the test-suite's tolerances (FP32 1e-5,
FP64 1e-12 relative), on two calls in a row, since each call reuses the array
the previous one left behind.  It always adds weight gradients into its FP64
chunk sums per tile, so the wide FP32 cases (whose plans accumulate a chunk's
tiles in FP32 first) also compare the two summation paths.  This file sorts last so that a run stopping at
the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(jet, spec, widths, prec, p, x, src):
    lib = jet.load()
    s, keep = jet._spec_struct(spec)
    needed = spec.closure()
    nd = (jet.JetChan * len(needed))()
    for i, al in enumerate(needed):
        for j, k in enumerate(al):
            nd[i].alpha[j] = k
    w = (ctypes.c_int32 * len(widths))(*widths)
    grad = torch.empty_like(p)
    loss = torch.empty((), dtype=torch.float64, device=p.device)
    used = ctypes.c_size_t()
    st = lib.jet_backward_params_noalloc(ctypes.byref(s), spec.d_in, len(widths) - 1, w, len(needed), nd,
                                         jet.PRECISIONS[prec], jet._ptr(p), jet._ptr(x), x.shape[0], jet._ptr(src),
                                         jet._ptr(grad), jet._ptr(loss),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(used))
    assert st == 0, lib.jet_last_error()
    assert 0 < used.value <= 8 << 20
    return grad, loss


def _rel(a, b):
    a = a.double().cpu().numpy().ravel()
    b = b.double().cpu().numpy().ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name,prec,N,tol", [("ks_2x64x5", "fp32", 5000, 1e-5),
                                              ("burgers_2x20x4", "fp64", 1000, 1e-12),
                                              ("helmholtz_3x256x8", "fp32", 700, 1e-5),
                                              ("ns_psi_3x128x6", "fp32", 300, 1e-5),
                                              # > 64 tiles per chunk: the plan's FP32 runs flush and restart
                                              ("ns_psi_3x128x6", "fp32", 100000, 1e-5)])
def test_noalloc_matches_plan_path_twice(name, prec, N, tol):
    from paper_2606_29702_gb300 import jet, specs
    from paper_2606_29702_gb300 import workloads as wl
    cfg = wl.WORKLOADS[name]
    sp = specs.by_name(cfg["family"], **cfg["coefs"])
    X = wl.points(cfg["domain"], N, 3)
    plan = jet.Plan(sp, cfg["widths"], prec)
    dt = plan.dtype
    p = torch.tensor(wl.pack(wl.xavier_layers(cfg["widths"], 2, bias_std=0.1)), dtype=dt, device="cuda")
    x = torch.tensor(X, dtype=dt, device="cuda")
    src = torch.tensor(specs.helmholtz_source(X), dtype=dt, device="cuda") if sp.has_source else None
    g_ref, l_ref, _ = plan.backward(p, x, src)
    for _ in range(2):
        g, l = _noalloc(jet, sp, cfg["widths"], prec, p, x, src)
        torch.cuda.synchronize()
        assert _rel(g, g_ref) <= tol
        assert abs(float(l) - float(l_ref)) <= tol * abs(float(l_ref))


def test_noalloc_rejects_oversized_shape():
    from paper_2606_29702_gb300 import jet, specs
    sp = specs.helmholtz()
    widths = [3] + [256] * 15 + [1]  # FP64: two weight copies + one gradient slice, about 22 MB
    lib = jet.load()
    s, keep = jet._spec_struct(sp)
    needed = sp.closure()
    nd = (jet.JetChan * len(needed))()
    for i, al in enumerate(needed):
        for j, k in enumerate(al):
            nd[i].alpha[j] = k
    w = (ctypes.c_int32 * len(widths))(*widths)
    dummy = torch.zeros(8, device="cuda")
    st = lib.jet_backward_params_noalloc(ctypes.byref(s), 3, len(widths) - 1, w, len(needed), nd,
                                         jet.PRECISIONS["fp64"], jet._ptr(dummy), jet._ptr(dummy), 10 ** 6,
                                         jet._ptr(dummy), jet._ptr(dummy), None, None, None)
    assert st == 3 and b"8 MiB" in lib.jet_last_error()
