"""Generate the per-closure jet algebra of the CUDA path (jet_closures_gen.h).

A *closure class* is a downward-closed set of multi-indices (the partial jet
of Sec. 2.2: the derivative states a residual needs plus the lower-order chain
that produces them).  For each class this script emits straight-line device
code, specialised at compile time, for

* ``compose``: the activation rule of the jet, a_alpha = sum over set
  partitions pi of alpha of phi^(|pi|)(z) prod_{B in pi} z_B -- the
  multivariate Faa di Bruno formula, of which Eq. 2 (first order) and Eq. 3
  (second order) are the first two cases and the higher orders follow
  recursively as Sec. 2.2 states;
* ``tangent``: its Jacobian-vector product da = (da/dz) v;
* ``adjoint``: its vector-Jacobian product zb = (da/dz)^T ab, the reverse
  sweep through the activation used by the parameter gradient.

phi = tanh, with p[k] = phi^(k)(z_0) supplied by ``tanh_derivs``.

The compiled classes are the generic full-order sets d1o4, d2o2 and d3o2, the
exact closure of every residual family in the package's ``specs.py`` (read at
build time, so a family added there gets its own class on the next build), and
the sets named in the environment variable JET_EXTRA_CLASSES
('d:alpha,alpha,...;...', e.g. '2:00,10,01,11').  A plan carries the smallest
compiled class that contains its closure.

Run: python gen_closures.py <out.h>   (the build does this).
"""

import importlib.util
import itertools
import os
import sys
from collections import OrderedDict

HERE = os.path.dirname(os.path.abspath(__file__))

# name -> (d, list of multi-indices); channel 0 is the value, channels are
# sorted by total order so the highest-order channels form the last block.
CLASSES = OrderedDict()


def _full(d, order):
    out = []
    for n in range(order + 1):
        for al in itertools.product(range(n + 1), repeat=d):
            if sum(al) == n:
                out.append(al)
    return out


def _sort(chans):
    return sorted(set(tuple(c) for c in chans), key=lambda a: (sum(a), tuple(-x for x in a)))


def _load_specs():
    """The package's residual-family table (specs.py), loaded by path: it is
    plain Python with no dependencies."""
    sp = importlib.util.spec_from_file_location("jet_specs_table", os.path.join(HERE, os.pardir, "specs.py"))
    mod = importlib.util.module_from_spec(sp)
    sp.loader.exec_module(mod)
    return mod


def _add(name, d, chans):
    """Register a channel set unless an identical one is already compiled."""
    chans = _sort(chans)
    for d2, c2 in CLASSES.values():
        if d2 == d and c2 == chans:
            return
    CLASSES[name] = (d, chans)


def _parse_extra(text):
    """JET_EXTRA_CLASSES: 'd:alpha,alpha,...;d:...' with alpha as digits, e.g.
    '2:00,10,01,11' adds the set {(0,0), (1,0), (0,1), (1,1)} (closed downward
    here)."""
    out = []
    for item in filter(None, (t.strip() for t in text.split(";"))):
        d, rest = item.split(":")
        d = int(d)
        chans = [tuple(int(ch) for ch in a.strip()) for a in rest.split(",") if a.strip()]
        if any(len(a) != d for a in chans):
            raise ValueError("JET_EXTRA_CLASSES: multi-index of the wrong length in %r" % item)
        out.append((d, _downward(chans, d)))
    return out


def _downward(chans, d):
    out, stack = set(), [tuple(a) for a in chans] + [tuple([0] * d)]
    while stack:
        a = stack.pop()
        if a in out:
            continue
        out.add(a)
        for i, k in enumerate(a):
            if k:
                stack.append(a[:i] + (k - 1,) + a[i + 1:])
    return sorted(out)


# Generic full-order sets (any residual up to that order in 1, 2 or 3
# coordinates), then the exact closure of every residual family of specs.py
# (Sec. 2.2: each residual carries exactly the channels it needs), then any
# sets named by the build environment.
CLASSES["d1o4"] = (1, _sort(_full(1, 4)))
CLASSES["d2o2"] = (2, _sort(_full(2, 2)))
CLASSES["d3o2"] = (3, _sort(_full(3, 2)))
_SPECS = _load_specs()
for _fam, _coefs in _SPECS.FAMILY_DEFAULTS.items():
    _s = _SPECS.by_name(_fam, **_coefs)
    _add(_fam, _s.d_in, _s.closure())
for _i, (_d, _chans) in enumerate(_parse_extra(os.environ.get("JET_EXTRA_CLASSES", ""))):
    _add("extra%d" % _i, _d, _chans)

# Tensor-core tile shapes compiled with compile-time constants (points per
# sub-tile, packed sub-tiles, 128-row halves, MMA width, CTA threads) besides
# the general kernel: the plans' built-in tile choices for the benchmarked
# networks of each class.  Other shapes and batches run the general kernel.
# A G of 0 leaves the packing to the work item: batches of members with widths
# 32, 64 and 128 and the same points per sub-tile (the ensemble) use it.  The
# launch takes the first entry that matches, so exact shapes come first.
FAST_SHAPES = {
    "burgers": [(64, 2, 1, 128, 512), (64, 0, 1, 128, 512)],  # width-64 nets (P = 128); ensembles, Pc = 64
    "ks": [(32, 2, 1, 128, 512), (40, 2, 1, 128, 512), (16, 2, 1, 128, 256)],  # BF16, BF16X3 P = 64, P = 80, 2 CTAs P = 32
    "helmholtz": [(16, 1, 2, 256, 512), (8, 1, 2, 256, 512)],  # 3->256x8->1: store P = 16, per tile P = 8
    "ns_psi": [(16, 1, 1, 128, 512), (8, 1, 1, 128, 512), (8, 1, 1, 128, 256)],  # BF16 16, BF16X3 8, 2 CTAs 8
    "ns_uvp": [(48, 2, 1, 128, 512)],                          # 2->64x6->3: P = 96
}


def set_partitions(items):
    if not items:
        yield []
        return
    first, rest = items[0], items[1:]
    for part in set_partitions(rest):
        yield [[first]] + part
        for i in range(len(part)):
            yield part[:i] + [[first] + part[i]] + part[i + 1:]


def fdb_terms(alpha, index):
    """Faa di Bruno terms of channel alpha: list of (coef, k, [block channel indices])."""
    d = len(alpha)
    coords = []
    for i, k in enumerate(alpha):
        coords += [i] * k
    acc = OrderedDict()
    for part in set_partitions(list(range(len(coords)))):
        blocks = []
        for blk in part:
            b = [0] * d
            for pos in blk:
                b[coords[pos]] += 1
            blocks.append(index[tuple(b)])
        key = (len(blocks), tuple(sorted(blocks)))
        acc[key] = acc.get(key, 0) + 1
    return [(c, k, list(bl)) for (k, bl), c in acc.items()]


def jacobian(chans):
    """J[a][b] = list of monomials (coef, pk, [z indices]) of d a_alpha / d z_beta."""
    index = {c: i for i, c in enumerate(chans)}
    C = len(chans)
    J = [[[] for _ in range(C)] for _ in range(C)]
    terms = {}
    for ai, al in enumerate(chans):
        if sum(al) == 0:
            terms[ai] = [(1, 0, [])]
        else:
            terms[ai] = fdb_terms(al, index)
        for coef, k, blocks in terms[ai]:
            # d/dz_0 acts through phi^(k)(z_0)
            J[ai][0].append((coef, k + 1, list(blocks)))
            for pos, b in enumerate(blocks):
                J[ai][b].append((coef, k, blocks[:pos] + blocks[pos + 1:]))
    # merge equal monomials (same phi order, same multiset of z factors)
    for ai in range(C):
        for bi in range(C):
            acc = OrderedDict()
            for coef, k, zs in J[ai][bi]:
                key = (k, tuple(sorted(zs)))
                acc[key] = acc.get(key, 0) + coef
            J[ai][bi] = [(c, k, list(zs)) for (k, zs), c in acc.items()]
    return terms, J


def mono(coef, k, zs, zname="z"):
    parts = ["p[%d]" % k] + ["%s[%d]" % (zname, i) for i in zs]
    s = "*".join(parts)
    if coef != 1:
        s = "T(%d)*%s" % (coef, s)
    return s


def factors(coef, k, zs):
    """Factor strings of one monomial coef * p[k] * prod z[zs]."""
    f = ["p[%d]" % k] + ["z[%d]" % i for i in zs]
    if coef != 1:
        f = ["T(%d)" % coef] + f
    return f


def fma_sum(terms):
    """Sum of products as a chain of fused multiply-adds: every term after the
    first adds as jfma(last factor, product of the others, partial sum); a
    first term is a plain product.  terms = lists of factor strings."""
    acc = None
    for fs in terms:
        if acc is None:
            acc = "*".join(fs)
        elif len(fs) == 1:
            acc = "(%s + %s)" % (acc, fs[0])
        else:
            acc = "jfma(%s, %s, %s)" % (fs[-1], "*".join(fs[:-1]), acc)
    return acc if acc is not None else "T(0)"


def emit_class(name, d, chans):
    C = len(chans)
    maxord = max(sum(c) for c in chans)
    terms, J = jacobian(chans)
    L = []
    L.append("struct Cls_%s {" % name)
    L.append("  static constexpr int D = %d;" % d)
    L.append("  static constexpr int C = %d;" % C)
    L.append("  static constexpr int MAXORD = %d;" % maxord)
    L.append("  static constexpr int NP = %d;  // p[0..MAXORD+1]" % (maxord + 2))
    first = []
    for i in range(d):
        e = tuple(int(j == i) for j in range(d))
        first.append(chans.index(e) if e in chans else -1)
    L.append("  // channel index of the first-order channel e_i (-1 if absent)")
    sel = " ".join("i == %d ? %d :" % (i, f) for i, f in enumerate(first)) + " -1"
    L.append("  static __host__ __device__ constexpr int first_order(int i) { return %s; }" % sel)
    L.append("  // first channel index of the highest derivative order")
    top = min(i for i, c in enumerate(chans) if sum(c) == maxord)
    L.append("  static constexpr int TOP_BEGIN = %d;" % top)
    # compose
    L.append("  template <class T> static __device__ __forceinline__ void compose(const T* z, const T* p, T* a) {")
    for ai in range(C):
        L.append("    a[%d] = %s;" % (ai, fma_sum([factors(c, k, bl) for c, k, bl in terms[ai]])))
    L.append("  }")
    # tangent
    L.append("  template <class T> static __device__ __forceinline__ void tangent(const T* z, const T* p, const T* v, T* da) {")
    for ai in range(C):
        parts = []
        for bi in range(C):
            if J[ai][bi]:
                parts.append([fma_sum([factors(c, k, zs) for c, k, zs in J[ai][bi]]), "v[%d]" % bi])
        L.append("    da[%d] = %s;" % (ai, fma_sum(parts)))
    L.append("  }")
    # adjoint
    L.append("  template <class T> static __device__ __forceinline__ void adjoint(const T* z, const T* p, const T* ab, T* zb) {")
    for bi in range(C):
        parts = []
        for ai in range(C):
            if J[ai][bi]:
                parts.append([fma_sum([factors(c, k, zs) for c, k, zs in J[ai][bi]]), "ab[%d]" % ai])
        L.append("    zb[%d] = %s;" % (bi, fma_sum(parts)))
    L.append("  }")
    L.append("};")
    return "\n".join(L)


def emit(path):
    out = []
    out.append("// Generated by gen_closures.py -- do not edit.")
    out.append("// Per-closure jet algebra: Faa di Bruno activation composition (Eq. 2-3 and")
    out.append("// their higher-order recursion, Sec. 2.2), its tangent and its adjoint.")
    out.append("#pragma once")
    out.append("")
    out.append("namespace jet {")
    out.append("")
    out.append("// fused multiply-add of the jet algebra; a packed type adds its own overload")
    out.append("__device__ __forceinline__ float jfma(float a, float b, float c) { return fmaf(a, b, c); }")
    out.append("__device__ __forceinline__ double jfma(double a, double b, double c) { return fma(a, b, c); }")
    out.append("")
    for name, (d, chans) in CLASSES.items():
        out.append("// %s: d=%d, channels %s" % (name, d, " ".join("".join(str(x) for x in c) for c in chans)))
        out.append(emit_class(name, d, chans))
        out.append("")
    # host table
    out.append("struct ClassInfo { const char* name; int d; int C; int maxord; unsigned char alpha[16][3]; };")
    out.append("static const ClassInfo kClassInfo[] = {")
    for name, (d, chans) in CLASSES.items():
        al = ", ".join("{%s}" % ", ".join(str(c[i]) if i < d else "0" for i in range(3)) for c in chans)
        out.append("  {\"%s\", %d, %d, %d, {%s}}," % (name, d, len(chans), max(sum(c) for c in chans), al))
    out.append("};")
    out.append("static constexpr int kNumClasses = %d;" % len(CLASSES))
    out.append("")
    out.append("template <int ID> struct ClassById;")
    for i, n in enumerate(CLASSES):
        out.append("template <> struct ClassById<%d> { using type = Cls_%s; };" % (i, n))
    out.append("")
    out.append("// per class id: JET_TC_SHAPES_<id>(M) expands M(PC, G, H, W, NT) for every compiled fixed shape")
    for i, n in enumerate(CLASSES):
        shapes = FAST_SHAPES.get(n, [])
        out.append("#define JET_TC_SHAPES_%d(M) %s" % (i, " ".join("M(%d, %d, %d, %d, %d)" % t for t in shapes)))
    out.append("")
    out.append("// X-macro over the classes: JET_FOR_EACH_CLASS(M) expands M(id, Cls_name)")
    out.append("#define JET_FOR_EACH_CLASS(M) \\")
    out.append(" \\\n".join("  M(%d, Cls_%s)" % (i, n) for i, n in enumerate(CLASSES)))
    out.append("")
    out.append("}  // namespace jet")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    emit(sys.argv[1] if len(sys.argv) > 1 else "jet_closures_gen.h")
