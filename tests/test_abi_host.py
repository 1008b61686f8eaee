"""Host-side checks of the C ABI (no GPU needed).

* libjet.so loads and exports every function include/jet.h declares;
* plan creation rejects bad shapes, non-closed channel sets and residuals that
  use channels outside the needed set before touching the device.
"""
import ctypes
import os
import re

import pytest

from paper_2606_29702_gb300 import jet, specs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "jet.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(jet_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = jet.load()
    names = _declared()
    assert "jet_plan_create" in names and "jet_train_step" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(jet.EXPORTS) == set(names)
    assert b"sm_103a" in lib.jet_version()


def _create(spec, widths, needed=None, prec="fp32", auto_close=False):
    lib = jet.load()
    s, keep = jet._spec_struct(spec)
    needed = spec.closure() if needed is None else needed
    nd = (jet.JetChan * max(1, len(needed)))()
    for i, al in enumerate(needed):
        for j, k in enumerate(al):
            nd[i].alpha[j] = k
    w = (ctypes.c_int32 * len(widths))(*widths)
    h = ctypes.c_void_p()
    st = lib.jet_plan_create(ctypes.byref(h), ctypes.byref(s), spec.d_in, len(widths) - 1, w, len(needed), nd,
                             jet.PRECISIONS[prec], 0, 1 if auto_close else 0)
    return st, lib.jet_last_error().decode()


def test_rejects_bad_shapes():
    sp = specs.burgers(0.01)
    assert _create(sp, [3, 20, 1])[0] == 1          # widths[0] != d_in
    assert _create(sp, [2, 22, 1])[0] == 3          # width not a multiple of 4
    assert _create(sp, [2, 512, 1])[0] == 3         # width above 256
    assert _create(sp, [2, 20])[0] == 1             # a single layer
    assert _create(sp, [2, 20, 20, 5])[0] == 1      # n_out above 4


def test_rejects_non_closed_needed_set():
    sp = specs.burgers(0.01)
    st, msg = _create(sp, [2, 20, 1], needed=[(0, 0), (0, 1), (2, 0)])  # u_x missing below u_xx
    assert st == 2 and "closed" in msg


def test_rejects_spec_outside_needed():
    sp = specs.ks()
    st, msg = _create(sp, [2, 16, 1], needed=[(0, 0), (1, 0), (0, 1), (2, 0)])
    assert st == 1 and "not in needed" in msg


def test_unsupported_closure():
    # fifth order in x is outside every compiled channel set
    sp = specs.Spec("x5", 2, 1, [[(1.0, [(0, (5, 0))])]])
    st, msg = _create(sp, [2, 16, 1], auto_close=True)
    assert st == 3


def _noalloc_status(spec_struct, d_in, widths, needed):
    """Status of jet_backward_params_noalloc for a spec the host checks must
    reject: the pointers are never dereferenced and no CUDA call is made."""
    lib = jet.load()
    nd = (jet.JetChan * max(1, len(needed)))()
    for i, al in enumerate(needed):
        for j, k in enumerate(al):
            nd[i].alpha[j] = k
    w = (ctypes.c_int32 * len(widths))(*widths)
    fake = ctypes.c_void_p(256)
    st = lib.jet_backward_params_noalloc(ctypes.byref(spec_struct), d_in, len(widths) - 1, w, len(needed), nd,
                                         jet.PRECISIONS["fp32"], fake, fake, 100, None, fake, None, None, None)
    return st, lib.jet_last_error().decode()


def test_noalloc_rejects_malformed_specs_on_the_host():
    sp = specs.burgers(0.01)
    needed = sp.closure()
    # a negative monomial count
    s, keep = jet._spec_struct(sp)
    s.n_mono[0] = -1
    st, msg = _noalloc_status(s, 2, [2, 20, 1], needed)
    assert st == 1 and "monomial list" in msg
    # a NULL monomial list with a positive count
    s, keep = jet._spec_struct(sp)
    s.mono[0] = ctypes.cast(None, ctypes.POINTER(jet.JetMonomial))
    st, msg = _noalloc_status(s, 2, [2, 20, 1], needed)
    assert st == 1 and "monomial list" in msg
    # a needed multi-index in a coordinate beyond d_in
    s, keep = jet._spec_struct(sp)
    st, msg = _noalloc_status(s, 2, [2, 20, 1], needed + [(0, 0, 1)])
    assert st == 1 and "coordinate >= d_in" in msg
    # a residual factor differentiating a coordinate beyond d_in
    bad = specs.Spec("bad", 2, 1, [[(1.0, [(0, (0, 0, 1))])]])
    s, keep = jet._spec_struct(bad)
    st, msg = _noalloc_status(s, 2, [2, 20, 1], needed)
    assert st == 1 and "coordinate >= d_in" in msg
