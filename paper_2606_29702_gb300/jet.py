"""Python binding of libjet (argument marshalling only).

Every step of the path runs in the CUDA library: this module converts torch
tensors to device pointers and calls the C ABI of ``include/jet.h`` with the
same names.  Importing it loads ``lib/libjet.so`` and raises if the library is
missing: there is no CPU fallback.
"""

import ctypes
import os

import torch

from . import specs as _specs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libjet.so")

PRECISIONS = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3, "bf16x3": 4}
FLAG_AUTO_CLOSE = 0x1
FLAG_STORE = 0x2
STATUS = {0: "JET_OK", 1: "JET_ERR_INVALID", 2: "JET_ERR_NOT_CLOSED", 3: "JET_ERR_UNSUPPORTED",
          4: "JET_ERR_OOM", 5: "JET_ERR_CUDA", 6: "JET_ERR_TIMEOUT"}


class JetError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class JetChan(ctypes.Structure):
    _fields_ = [("out", ctypes.c_int32), ("alpha", ctypes.c_uint8 * 4)]


class JetMonomial(ctypes.Structure):
    _fields_ = [("coef", ctypes.c_double), ("n_fac", ctypes.c_int32), ("fac", JetChan * 4)]


class JetResidualSpec(ctypes.Structure):
    _fields_ = [("n_res", ctypes.c_int32), ("n_mono", ctypes.POINTER(ctypes.c_int32)),
                ("mono", ctypes.POINTER(ctypes.POINTER(JetMonomial))), ("has_source", ctypes.c_int32)]


class JetLossTerm(ctypes.Structure):
    _fields_ = [("spec", ctypes.POINTER(JetResidualSpec)), ("weight", ctypes.c_double), ("paired", ctypes.c_int32)]


class JetPlanInfo(ctypes.Structure):
    _fields_ = [("d_in", ctypes.c_int32), ("n_out", ctypes.c_int32), ("n_layers", ctypes.c_int32),
                ("n_channels", ctypes.c_int32), ("closure_class", ctypes.c_int32),
                ("class_name", ctypes.c_char * 32), ("n_params", ctypes.c_int64), ("precision", ctypes.c_int32),
                ("store_mode", ctypes.c_int32), ("store_max_points", ctypes.c_int64),
                ("tile_points", ctypes.c_int32), ("grid_ctas", ctypes.c_int32), ("workspace_bytes", ctypes.c_size_t),
                ("ctas_per_sm", ctypes.c_int32), ("cta_threads", ctypes.c_int32),
                ("wgrad_chunk_fp32", ctypes.c_int32)]


EXPORTS = ["jet_plan_create", "jet_plan_create_loss", "jet_plan_set_term_points", "jet_plan_get_info", "jet_forward_residual", "jet_backward_params", "jet_train_step",
           "jet_train_step_dev", "jet_plan_destroy", "jet_batch_create", "jet_batch_backward", "jet_batch_train_step",
           "jet_batch_train_step_dev", "jet_batch_destroy",
           "jet_debug_activation", "jet_plan_profile", "jet_plan_profile_read", "jet_backward_params_noalloc",
           "jet_debug_wait_timeout", "jet_last_error", "jet_version"]

_lib = None


def load():
    """Load libjet.so (built by paper_2606_29702_gb300.build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libjet.so not found at %s: run __graft_entry__.build() first" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    L.jet_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(JetResidualSpec), i32, i32,
                                  ctypes.POINTER(i32), i32, ctypes.POINTER(JetChan), i32, sz, i32]
    L.jet_plan_create_loss.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(JetLossTerm), i32, i32,
                                       ctypes.POINTER(i32), i32, ctypes.POINTER(JetChan), i32, sz, i32]
    L.jet_plan_set_term_points.argtypes = [vp, ctypes.POINTER(i64)]
    L.jet_plan_get_info.argtypes = [vp, ctypes.POINTER(JetPlanInfo)]
    L.jet_forward_residual.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp]
    L.jet_backward_params.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp, vp]
    L.jet_train_step.argtypes = [vp, vp, vp, vp, i64, ctypes.c_float, vp, i64, vp, vp, vp]
    L.jet_train_step_dev.argtypes = [vp, vp, vp, vp, vp, ctypes.c_float, vp, i64, vp, vp, vp]
    L.jet_plan_destroy.argtypes = [vp]
    L.jet_batch_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp), i32]
    L.jet_batch_backward.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i64),
                                     ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp]
    L.jet_batch_train_step.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), i64,
                                       ctypes.c_float, ctypes.POINTER(vp), ctypes.POINTER(i64), ctypes.POINTER(vp),
                                       vp, vp]
    L.jet_batch_train_step_dev.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), vp,
                                           ctypes.c_float, ctypes.POINTER(vp), ctypes.POINTER(i64),
                                           ctypes.POINTER(vp), vp, vp]
    L.jet_batch_destroy.argtypes = [vp]
    L.jet_debug_activation.argtypes = [vp, i32, i64, vp, vp, vp, vp]
    L.jet_backward_params_noalloc.argtypes = [ctypes.POINTER(JetResidualSpec), i32, i32, ctypes.POINTER(i32), i32,
                                              ctypes.POINTER(JetChan), i32, vp, vp, i64, vp, vp, vp, vp,
                                              ctypes.POINTER(sz)]
    L.jet_debug_wait_timeout.argtypes = [i64]
    L.jet_plan_profile.argtypes = [vp, i32]
    L.jet_plan_profile_read.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double)]
    L.jet_last_error.restype = ctypes.c_char_p
    L.jet_version.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("jet_last_error", "jet_version"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(st):
    if st != 0:
        raise JetError(st, load().jet_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _spec_struct(spec):
    """Keep-alive tuple of ctypes objects describing ``spec`` (a specs.Spec)."""
    n_res = spec.n_res
    arrays = []
    for comp in spec.components:
        arr = (JetMonomial * max(1, len(comp)))()
        for m, (coef, facs) in enumerate(comp):
            arr[m].coef = float(coef)
            arr[m].n_fac = len(facs)
            for f, (o, al) in enumerate(facs):
                arr[m].fac[f].out = o
                for i, k in enumerate(al):
                    arr[m].fac[f].alpha[i] = k
        arrays.append(arr)
    n_mono = (ctypes.c_int32 * n_res)(*[len(c) for c in spec.components])
    ptrs = (ctypes.POINTER(JetMonomial) * n_res)(*[ctypes.cast(a, ctypes.POINTER(JetMonomial)) for a in arrays])
    s = JetResidualSpec(n_res, n_mono, ptrs, 1 if spec.has_source else 0)
    return s, (arrays, n_mono, ptrs)


class Plan:
    """A libjet plan: one residual on one network shape at one precision."""

    def __init__(self, spec, widths, precision="fp32", needed=None, mem_budget=0, store=False, auto_close=True,
                 tile=None, ctas=0):
        L = load()
        self.tile = tile
        self.ctas = ctas
        self.spec = spec
        self.widths = list(widths)
        self.precision = precision
        s, keep = _spec_struct(spec)
        needed = spec.closure() if needed is None else needed
        nd = (JetChan * max(1, len(needed)))()
        for i, al in enumerate(needed):
            for j, k in enumerate(al):
                nd[i].alpha[j] = k
        w = (ctypes.c_int32 * len(widths))(*widths)
        flags = (FLAG_AUTO_CLOSE if auto_close else 0) | (FLAG_STORE if store else 0)
        if tile:
            if tile % 8 or not 8 <= tile <= 2040:
                raise ValueError("tile must be a multiple of 8 in [8, 2040]")
            flags |= (tile // 8) << 8
        if ctas not in (0, 1, 2):
            raise ValueError("ctas must be 0 (plan's choice), 1 or 2")
        flags |= ctas << 16
        h = ctypes.c_void_p()
        _check(L.jet_plan_create(ctypes.byref(h), ctypes.byref(s), spec.d_in, len(widths) - 1, w, len(needed), nd,
                                 PRECISIONS[precision], int(mem_budget), flags))
        self._h = h
        self._keep = keep
        self.dtype = torch.float64 if precision == "fp64" else torch.float32

    @property
    def handle(self):
        return self._h

    def info(self):
        inf = JetPlanInfo()
        _check(load().jet_plan_get_info(self._h, ctypes.byref(inf)))
        d = {k: getattr(inf, k) for k, _ in JetPlanInfo._fields_}
        d["class_name"] = d["class_name"].decode()
        return d

    def _chk(self, t, name, shape=None):
        if t is None:
            return
        if not t.is_cuda or t.dtype != self.dtype or not t.is_contiguous():
            raise ValueError("%s must be a contiguous CUDA %s tensor" % (name, self.dtype))
        if shape is not None and tuple(t.shape) != tuple(shape):
            raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))

    def forward(self, params, X, source=None, want_r=True, stream=None):
        """(r [N, n_res] or None, loss (float64 scalar tensor)) -- jet_forward_residual."""
        N = X.shape[0]
        self._chk(params, "params")
        self._chk(X, "X", (N, self.spec.d_in))
        self._chk(source, "source", (N, self.spec.n_res))
        r = torch.empty((N, self.spec.n_res), dtype=self.dtype, device=X.device) if want_r else None
        loss = torch.empty((), dtype=torch.float64, device=X.device)
        _check(load().jet_forward_residual(self._h, _ptr(params), _ptr(X), N, _ptr(source), _ptr(r), _ptr(loss),
                                           _stream(stream)))
        return r, loss

    def backward(self, params, X, source=None, want_r=False, stream=None):
        """(grad packed like params, loss, r or None) -- jet_backward_params."""
        N = X.shape[0]
        self._chk(params, "params")
        self._chk(X, "X", (N, self.spec.d_in))
        self._chk(source, "source", (N, self.spec.n_res))
        grad = torch.empty_like(params)
        loss = torch.empty((), dtype=torch.float64, device=X.device)
        r = torch.empty((N, self.spec.n_res), dtype=self.dtype, device=X.device) if want_r else None
        _check(load().jet_backward_params(self._h, _ptr(params), _ptr(X), N, _ptr(source), _ptr(grad), _ptr(r),
                                          _ptr(loss), _stream(stream)))
        return grad, loss, r

    def train_step(self, params, m, v, step, lr, X, source=None, loss=None, stream=None):
        """In-place Adam step on params (jet_train_step); returns the pre-step loss tensor."""
        N = X.shape[0]
        for t, nme in ((params, "params"), (m, "adam_m"), (v, "adam_v")):
            self._chk(t, nme)
        self._chk(X, "X", (N, self.spec.d_in))
        if loss is None:
            loss = torch.empty((), dtype=torch.float64, device=X.device)
        _check(load().jet_train_step(self._h, _ptr(params), _ptr(m), _ptr(v), int(step), float(lr), _ptr(X), N,
                                     _ptr(source), _ptr(loss), _stream(stream)))
        return loss

    def train_step_dev(self, params, m, v, step_counter, lr, X, source=None, loss=None, stream=None):
        """In-place Adam step with a device step counter (jet_train_step_dev):
        ``step_counter`` is a CUDA int64 tensor holding the steps already
        taken; the call advances it on the device."""
        N = X.shape[0]
        for t, nme in ((params, "params"), (m, "adam_m"), (v, "adam_v")):
            self._chk(t, nme)
        self._chk(X, "X", (N, self.spec.d_in))
        _chk_counter(step_counter)
        if loss is None:
            loss = torch.empty((), dtype=torch.float64, device=X.device)
        _check(load().jet_train_step_dev(self._h, _ptr(params), _ptr(m), _ptr(v), _ptr(step_counter), float(lr),
                                         _ptr(X), N, _ptr(source), _ptr(loss), _stream(stream)))
        return loss

    def debug_activation(self, kind, z, v=None, stream=None):
        out = torch.empty_like(z)
        _check(load().jet_debug_activation(self._h, int(kind), z.shape[0], _ptr(z), _ptr(v), _ptr(out),
                                           _stream(stream)))
        return out

    def profile(self, enable=True):
        _check(load().jet_plan_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        """(launches, summed device ms) of the dominant kernel since the last read."""
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        _check(load().jet_plan_profile_read(self._h, ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.jet_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _chk_counter(t):
    if not t.is_cuda or t.dtype != torch.int64 or t.numel() != 1:
        raise ValueError("step_counter must be a one-element CUDA int64 tensor")


class _LossShape:
    """What the call checks of a Plan read from its spec, for a composite loss."""

    def __init__(self, terms):
        specs = [t[0] for t in terms]
        self.name = "+".join(sp.name for sp in specs)
        self.d_in = specs[0].d_in
        self.n_out = specs[0].n_out
        self.n_res = max(sp.n_res for sp in specs)
        self.has_source = any(sp.has_source for sp in specs)
        self._specs = specs

    def closure(self):
        out = set()
        for sp in self._specs:
            out |= set(sp.closure())
        return sorted(out, key=lambda a: (sum(a), a))


class LossPlan(Plan):
    """A composite-loss plan (jet_plan_create_loss): ``terms`` is a list of
    (spec, weight, paired) in point order; ``set_term_points`` (or the
    ``counts`` argument of the calls) gives each term's number of points."""

    def __init__(self, terms, widths, precision="fp32", needed=None, mem_budget=0, store=False, tile=None, ctas=0):
        L = load()
        self.tile = tile
        self.ctas = ctas
        self.spec = _LossShape(terms)
        self.widths = list(widths)
        self.precision = precision
        structs = [_spec_struct(t[0]) for t in terms]
        arr = (JetLossTerm * len(terms))()
        for i, ((sp, w, paired), (s, _)) in enumerate(zip(terms, structs)):
            arr[i].spec = ctypes.pointer(s)
            arr[i].weight = float(w)
            arr[i].paired = 1 if paired else 0
        needed = self.spec.closure() if needed is None else needed
        nd = (JetChan * max(1, len(needed)))()
        for i, al in enumerate(needed):
            for j, k in enumerate(al):
                nd[i].alpha[j] = k
        wd = (ctypes.c_int32 * len(widths))(*widths)
        flags = FLAG_AUTO_CLOSE | (FLAG_STORE if store else 0) | ((tile // 8) << 8 if tile else 0) | (ctas << 16)
        h = ctypes.c_void_p()
        _check(L.jet_plan_create_loss(ctypes.byref(h), len(terms), arr, self.spec.d_in, len(widths) - 1, wd,
                                      len(needed), nd, PRECISIONS[precision], int(mem_budget), flags))
        self._h = h
        self._keep = (structs, arr)
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.counts = None

    def set_term_points(self, counts):
        c = (ctypes.c_int64 * len(counts))(*[int(x) for x in counts])
        _check(load().jet_plan_set_term_points(self._h, c))
        self.counts = list(counts)


def _vp_array(ts):
    return (ctypes.c_void_p * len(ts))(*[None if t is None else t.data_ptr() for t in ts])


class Batch:
    """Many plans run as one persistent launch (jet_batch_*)."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(plans))(*[p.handle.value for p in plans])
        h = ctypes.c_void_p()
        _check(load().jet_batch_create(ctypes.byref(h), len(plans), arr, 0))
        self._h = h

    def backward(self, params, X, sources=None, stream=None):
        n = len(self.plans)
        grads = [torch.empty_like(p) for p in params]
        loss = torch.empty(n, dtype=torch.float64, device=X[0].device)
        Ns = (ctypes.c_int64 * n)(*[x.shape[0] for x in X])
        src = _vp_array(sources) if sources is not None else None
        _check(load().jet_batch_backward(self._h, _vp_array(params), _vp_array(X), Ns, src, _vp_array(grads),
                                         _ptr(loss), _stream(stream)))
        return grads, loss

    def train_step(self, params, m, v, step, lr, X, sources=None, loss=None, stream=None):
        n = len(self.plans)
        if loss is None:
            loss = torch.empty(n, dtype=torch.float64, device=X[0].device)
        Ns = (ctypes.c_int64 * n)(*[x.shape[0] for x in X])
        src = _vp_array(sources) if sources is not None else None
        _check(load().jet_batch_train_step(self._h, _vp_array(params), _vp_array(m), _vp_array(v), int(step),
                                           float(lr), _vp_array(X), Ns, src, _ptr(loss), _stream(stream)))
        return loss

    def train_step_dev(self, params, m, v, step_counter, lr, X, sources=None, loss=None, stream=None):
        """Batched Adam step with one device step counter (jet_batch_train_step_dev)."""
        n = len(self.plans)
        _chk_counter(step_counter)
        if loss is None:
            loss = torch.empty(n, dtype=torch.float64, device=X[0].device)
        Ns = (ctypes.c_int64 * n)(*[x.shape[0] for x in X])
        src = _vp_array(sources) if sources is not None else None
        _check(load().jet_batch_train_step_dev(self._h, _vp_array(params), _vp_array(m), _vp_array(v),
                                               _ptr(step_counter), float(lr), _vp_array(X), Ns, src, _ptr(loss),
                                               _stream(stream)))
        return loss

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.jet_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class JetResidual(torch.autograd.Function):
    """(r, loss) = JetResidual.apply(params, X, plan, source).

    Forward runs jet_forward_residual; backward runs jet_backward_params and
    returns dL/dparams scaled by the loss cotangent.  Only the scalar loss may
    carry a cotangent: the reverse sweep is the adjoint of the mean-squared
    residual loss (Sec. 3.1.1), not of an arbitrary function of r.
    """

    @staticmethod
    def forward(ctx, params, X, plan, source=None):
        r, loss = plan.forward(params, X, source)
        ctx.plan = plan
        ctx.save_for_backward(params, X, source if source is not None else torch.empty(0, device=X.device))
        ctx.has_source = source is not None
        ctx.mark_non_differentiable(r)
        return r, loss

    @staticmethod
    def backward(ctx, g_r, g_loss):
        params, X, source = ctx.saved_tensors
        if g_r is not None and bool(torch.any(g_r != 0)):
            raise RuntimeError("JetResidual: only the loss output can be differentiated")
        grad, _, _ = ctx.plan.backward(params, X, source if ctx.has_source else None)
        return grad * g_loss.to(grad.dtype), None, None, None


def plan_for(name, widths, precision="fp32", **coefs):
    """Convenience: a plan for a named PDE family of ``specs``."""
    return Plan(_specs.by_name(name, **coefs), widths, precision)


def debug_wait_timeout(budget_ns=1_000_000):
    """Status of jet_debug_wait_timeout (JET_ERR_TIMEOUT == 6 when the bounded wait works)."""
    L = load()
    return L.jet_debug_wait_timeout(int(budget_ns))
