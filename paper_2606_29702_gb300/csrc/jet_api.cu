// Host side of libjet: plan creation (closure of the needed multi-indices,
// choice of the compiled channel set, tiling, workspace), call orchestration
// and the batched-ensemble work list.  See include/jet.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <vector>

#include "../../include/jet.h"
#include "jet_closures_gen.h"
#include "jet_internal.h"
#include "jet_plan.h"
#include "jet_tc.h"

using namespace jet;

namespace {

thread_local std::string g_err;

jet_status fail(jet_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

jet_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? JET_ERR_OOM : JET_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(expr)                                   \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr); \
  } while (0)

using Alpha = std::vector<int>;  // orders per coordinate, length d

cudaError_t simt_launch(int cls, bool fp64, const SimtArgs& a, int grid, size_t smem, cudaStream_t s) {
  switch (cls) {
#define CASE(id, cl) \
  case id:           \
    return simt_launch_id<id>(fp64, a, grid, smem, s);
    JET_FOR_EACH_CLASS(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t simt_occupancy(int cls, bool fp64, size_t smem, int* blocks) {
  switch (cls) {
#define CASE(id, cl) \
  case id:           \
    return simt_max_active_id<id>(fp64, smem, blocks);
    JET_FOR_EACH_CLASS(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t debug_act(int cls, int kind, long long n, const double* z, const double* v, double* out, cudaStream_t s) {
  switch (cls) {
#define CASE(id, cl) \
  case id:           \
    return debug_activation_id<id>(kind, n, z, v, out, s);
    JET_FOR_EACH_CLASS(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

}  // namespace

void jet::set_last_error(const char* msg) { g_err = msg; }

void jet::plan_prof_begin(jet_plan_s* p, cudaStream_t s) {
  if (!p->profiling) return;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, s);
  p->prof.push_back({a, b});
}

void jet::plan_prof_end(jet_plan_s* p, cudaStream_t s) {
  if (!p->profiling || p->prof.empty()) return;
  cudaEventRecord(p->prof.back().second, s);
}

// Record an event pair around the dominant kernel of a call when profiling.
struct ProfScope {
  jet_plan_s* p;
  cudaStream_t s;
  ProfScope(jet_plan_s* p_, cudaStream_t s_) : p(p_), s(s_) { jet::plan_prof_begin(p, s); }
  ~ProfScope() { jet::plan_prof_end(p, s); }
};

namespace {

void free_plan_ws(jet_plan_s* p) {
  for (auto& e : p->prof) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  p->prof.clear();
  cudaFree(p->Wt);
  cudaFree(p->grad_slices);
  cudaFree(p->loss_slices);
  cudaFree(p->scratch);
  cudaFree(p->store);
  p->Wt = p->grad_slices = p->loss_slices = nullptr;
  p->scratch = p->store = nullptr;
  if (p->tcp) tc_plan_destroy(p->tcp);
  p->tcp = nullptr;
}

bool alpha_leq(const Alpha& a, const Alpha& b) {
  for (size_t i = 0; i < a.size(); ++i)
    if (a[i] > b[i]) return false;
  return true;
}

// all multi-indices below a (componentwise), including a and 0
void below(const Alpha& a, std::set<Alpha>& out) {
  Alpha cur(a.size(), 0);
  while (true) {
    out.insert(cur);
    size_t i = 0;
    while (i < a.size()) {
      if (cur[i] < a[i]) {
        ++cur[i];
        break;
      }
      cur[i] = 0;
      ++i;
    }
    if (i == a.size()) break;
  }
}

int tile_points(int wmax, bool fp64) {
  const int TP = fp64 ? 2 : 4;
  int q = kSimtThreads / wmax;
  if (q < 1) q = 1;
  return TP * q;
}

int pitch_for(int cols, bool fp64) {
  // rows are offset by 16 bytes modulo 128: conflict-free 16-byte accesses
  // by lanes that walk consecutive rows
  const int mod = fp64 ? 16 : 32, want = fp64 ? 2 : 4;
  int p = cols;
  while (p % mod != want) ++p;
  return p;
}

size_t smem_bytes(int C, int P, int pitch, int wmax, int n_out, int d, size_t elem) {
  return simt_smem_bytes(C, P, pitch, wmax, n_out, d, elem);
}

}  // namespace

extern "C" {

const char* jet_last_error(void) { return g_err.c_str(); }

const char* jet_version(void) { return "libjet 0.1 (sm_103a)"; }

}  // extern "C"

// Plan creation for one residual (n_specs = 1, grouped = false: the loss is
// the mean over all N points) or for a composite loss of n_specs terms, each
// over its own block of points (grouped = true).
static jet_status plan_create(jet_plan_t* out, int n_specs, const jet_residual_spec* const* specs,
                              const double* weights, const int32_t* paired, bool grouped, int32_t d_in,
                              int32_t n_layers, const int32_t* widths, int32_t n_needed, const jet_chan* needed,
                              jet_precision prec, size_t mem_budget_bytes, int32_t flags) {
  if (!out) return fail(JET_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!specs || !widths || (n_needed > 0 && !needed)) return fail(JET_ERR_INVALID, "NULL spec, widths or needed");
  for (int g = 0; g < n_specs; ++g)
    if (!specs[g]) return fail(JET_ERR_INVALID, "NULL residual spec of loss term %d", g);
  if (d_in < 1 || d_in > 3) return fail(JET_ERR_INVALID, "d_in must be 1..3 (got %d)", d_in);
  if (n_layers < 2 || n_layers > kMaxLayers) return fail(JET_ERR_INVALID, "n_layers must be 2..%d", kMaxLayers);
  if (widths[0] != d_in) return fail(JET_ERR_INVALID, "widths[0] (%d) != d_in (%d)", widths[0], d_in);
  const int n_out = widths[n_layers];
  if (n_out < 1 || n_out > kMaxOut) return fail(JET_ERR_INVALID, "n_out must be 1..%d", kMaxOut);
  for (int l = 1; l < n_layers; ++l)
    if (widths[l] < 4 || widths[l] > 256 || widths[l] % 4)
      return fail(JET_ERR_UNSUPPORTED, "hidden width %d: must be a multiple of 4 in [4, 256]", widths[l]);
  if (prec < JET_FP64 || prec > JET_BF16X3) return fail(JET_ERR_INVALID, "unknown precision %d", (int)prec);
  for (int g = 0; g < n_specs; ++g) {
    const jet_residual_spec* spec = specs[g];
    if (spec->n_res < 1 || spec->n_res > kMaxRes || !spec->n_mono || !spec->mono)
      return fail(JET_ERR_INVALID, "residual spec: n_res must be 1..%d with n_mono and mono set", kMaxRes);
  }

  // ---- channel closure (Sec. 2.2: required states plus their lower-order chain)
  std::set<Alpha> need;
  for (int i = 0; i < n_needed; ++i) {
    Alpha a(d_in);
    for (int j = 0; j < d_in; ++j) a[j] = needed[i].alpha[j];
    for (int j = d_in; j < 4; ++j)
      if (needed[i].alpha[j]) return fail(JET_ERR_INVALID, "needed[%d] differentiates a coordinate >= d_in", i);
    need.insert(a);
  }
  need.insert(Alpha(d_in, 0));
  std::set<Alpha> closure;
  for (const Alpha& a : need) below(a, closure);
  if (!(flags & JET_FLAG_AUTO_CLOSE) && closure.size() != need.size())
    return fail(JET_ERR_NOT_CLOSED, "needed multi-indices are not downward closed (%zu given, closure has %zu)",
                need.size(), closure.size());
  // every spec factor must be carried
  int n_terms = 0;
  for (int g = 0; g < n_specs; ++g) {
    const jet_residual_spec* spec = specs[g];
    for (int c = 0; c < spec->n_res; ++c) {
      if (spec->n_mono[c] < 0 || (spec->n_mono[c] > 0 && !spec->mono[c]))
        return fail(JET_ERR_INVALID, "residual component %d: bad monomial list", c);
      n_terms += spec->n_mono[c];
    }
  }
  if (n_terms > kMaxTerms) return fail(JET_ERR_UNSUPPORTED, "%d monomials > %d", n_terms, kMaxTerms);
  for (int g = 0; g < n_specs; ++g) {
    const jet_residual_spec* spec = specs[g];
    for (int c = 0; c < spec->n_res; ++c)
      for (int m = 0; m < spec->n_mono[c]; ++m) {
        const jet_monomial& mo = spec->mono[c][m];
        if (mo.n_fac < 0 || mo.n_fac > 4) return fail(JET_ERR_INVALID, "monomial with %d factors", mo.n_fac);
        for (int f = 0; f < mo.n_fac; ++f) {
          const int o = mo.fac[f].out & ~JET_PAIR_SECOND;
          if ((mo.fac[f].out & JET_PAIR_SECOND) && !(paired && paired[g]))
            return fail(JET_ERR_INVALID, "JET_PAIR_SECOND in a term that is not paired");
          if (o < 0 || o >= n_out) return fail(JET_ERR_INVALID, "monomial factor output %d out of range", o);
          Alpha a(d_in);
          for (int j = 0; j < d_in; ++j) a[j] = mo.fac[f].alpha[j];
          for (int j = d_in; j < 4; ++j)
            if (mo.fac[f].alpha[j]) return fail(JET_ERR_INVALID, "a residual factor differentiates a coordinate >= d_in");
          if (!closure.count(a)) return fail(JET_ERR_INVALID, "residual uses a multi-index that is not in needed");
        }
      }
  }
  // ---- smallest compiled channel set containing the closure
  int best = -1;
  for (int k = 0; k < kNumClasses; ++k) {
    const ClassInfo& ci = kClassInfo[k];
    if (ci.d != d_in) continue;
    std::set<Alpha> have;
    for (int c = 0; c < ci.C; ++c) {
      Alpha a(d_in);
      for (int j = 0; j < d_in; ++j) a[j] = ci.alpha[c][j];
      have.insert(a);
    }
    bool ok = true;
    for (const Alpha& a : closure) ok = ok && have.count(a);
    if (ok && (best < 0 || ci.C < kClassInfo[best].C)) best = k;
  }
  if (best < 0) return fail(JET_ERR_UNSUPPORTED, "no compiled channel set in %d coordinates contains the closure", d_in);

  jet_plan_s* p = new jet_plan_s();
  cudaGetDevice(&p->device);
  p->d = d_in;
  p->L = n_layers;
  p->n_out = n_out;
  p->n_res = 0;
  for (int g = 0; g < n_specs; ++g) p->n_res = std::max(p->n_res, (int)specs[g]->n_res);
  p->widths.assign(widths, widths + n_layers + 1);
  p->cls = best;
  p->C = kClassInfo[best].C;
  p->prec = prec;
  p->fp64 = prec == JET_FP64;
  p->tc = prec >= JET_TF32;
  p->elem = p->fp64 ? 8 : 4;
  p->has_source = false;
  for (int g = 0; g < n_specs; ++g) p->has_source = p->has_source || specs[g]->has_source != 0;
  auto chan_index = [&](const jet_chan& ch) {
    const ClassInfo& ci = kClassInfo[best];
    for (int c = 0; c < ci.C; ++c) {
      bool eq = true;
      for (int j = 0; j < d_in; ++j) eq = eq && ci.alpha[c][j] == ch.alpha[j];
      if (eq) return c;
    }
    return -1;
  };
  for (int g = 0; g < n_specs; ++g) {
    const jet_residual_spec* spec = specs[g];
    DevGroup G;
    memset(&G, 0, sizeof(G));
    G.t0 = (int)p->terms.size();
    for (int c = 0; c < spec->n_res; ++c)
      for (int m = 0; m < spec->n_mono[c]; ++m) {
        const jet_monomial& mo = spec->mono[c][m];
        DevTerm t;
        t.coef = mo.coef;
        t.comp = c;
        t.nfac = mo.n_fac;
        t.pmask = 0;
        for (int f = 0; f < 4; ++f) t.fac[f] = 0;
        for (int f = 0; f < mo.n_fac; ++f) {
          t.fac[f] = (mo.fac[f].out & ~JET_PAIR_SECOND) * p->C + chan_index(mo.fac[f]);
          if (mo.fac[f].out & JET_PAIR_SECOND) t.pmask |= 1 << f;
        }
        p->terms.push_back(t);
      }
    G.t1 = (int)p->terms.size();
    G.n_res = spec->n_res;
    G.paired = paired && paired[g] ? 1 : 0;
    G.has_source = spec->has_source != 0;
    G.scale = weights ? weights[g] : 1.0;  // the term's weight; divided by its residual count per call
    p->groups.push_back(G);
  }
  p->n_groups = grouped ? n_specs : 0;
  long long off = 0;
  for (int l = 0; l < n_layers; ++l) {
    p->off_W.push_back(off);
    off += (long long)widths[l] * widths[l + 1];
    p->off_b.push_back(off);
    off += widths[l + 1];
  }
  p->n_params = off;

  // ---- tiling and occupancy of the fused SIMT kernel
  int wmax = 0;
  for (int l = 1; l < n_layers; ++l) wmax = std::max(wmax, widths[l]);
  const int p8 = JET_FLAG_TILE_GET(flags);
  p->P = p8 ? 8 * p8 : tile_points(wmax, p->fp64);
  p->S = simt_point_stride(p->C, p->P);
  p->pitch = pitch_for(p->S * p->P, p->fp64);
  p->smem = smem_bytes(p->C, p->P, p->pitch, wmax, n_out, d_in, p->elem);
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, p->device);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cudaGetDeviceProperties");
  }
  int per_sm = 0;
  if (!p->tc) {
    e = simt_occupancy(p->cls, p->fp64, p->smem, &per_sm);
    if (e != cudaSuccess || per_sm < 1) {
      delete p;
      return e != cudaSuccess ? cuda_fail(e, "occupancy") : fail(JET_ERR_UNSUPPORTED, "SIMT tile does not fit one SM");
    }
    p->grid = prop.multiProcessorCount * per_sm;
    p->ctas_per_sm = per_sm;
  }

  // ---- workspace
  long long jet_elems = 0;  // hidden z-jets of one tile
  for (int l = 1; l < n_layers; ++l) jet_elems += (long long)p->C * p->P * widths[l];
  if (!p->tc) {
    // FP32 forms whose per-chunk FP64 slices would not stay in L2 add the
    // hidden-layer weight gradients of a chunk in an FP32 accumulator and
    // flush once per chunk; otherwise per-tile FP64 adds into L2-resident
    // slices are the cheaper of the two
    const bool slices_fit = (double)p->grid * p->n_params * sizeof(double) <= kSimtSliceL2Bytes;
    const long long wacc = slices_fit ? 0 : simt_wacc_elems(widths, n_layers, p->fp64);
    p->scratch_stride = jet_elems + wacc;
    p->wacc_off = wacc ? jet_elems : -1;
    size_t b_wt = (size_t)weight_ws_elems(p->n_params) * p->elem;
    size_t b_gs = (size_t)p->grid * p->n_params * sizeof(double);
    size_t b_ls = (size_t)p->grid * sizeof(double);
    size_t b_sc = (size_t)p->grid * p->scratch_stride * p->elem;
    e = cudaMalloc(&p->Wt, b_wt);
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->grad_slices, b_gs);
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->loss_slices, b_ls);
    if (e == cudaSuccess) e = cudaMalloc(&p->scratch, b_sc);
    p->ws_bytes = b_wt + b_gs + b_ls + b_sc;
    if (e == cudaSuccess && (flags & JET_FLAG_STORE) && mem_budget_bytes > 0) {
      const size_t per_tile = (size_t)jet_elems * p->elem;
      long long tiles = (long long)(mem_budget_bytes / per_tile);
      if (tiles > 0) {
        p->store_tile_stride = jet_elems;
        p->store_max_points = tiles * p->P;
        e = cudaMalloc(&p->store, tiles * per_tile);
        p->ws_bytes += tiles * per_tile;
      }
    }
    if (e != cudaSuccess) {
      free_plan_ws(p);
      delete p;
      return cuda_fail(e, "workspace allocation");
    }
  } else {
    jet_status st = tc_plan_create(p, &p->tcp, prop, mem_budget_bytes, flags);
    if (st != JET_OK) {
      free_plan_ws(p);
      delete p;
      return st;
    }
  }
  *out = p;
  return JET_OK;
}

extern "C" {

jet_status jet_plan_create(jet_plan_t* out, const jet_residual_spec* spec, int32_t d_in, int32_t n_layers,
                           const int32_t* widths, int32_t n_needed, const jet_chan* needed, jet_precision prec,
                           size_t mem_budget_bytes, int32_t flags) {
  if (!spec) {
    if (out) *out = nullptr;
    return fail(JET_ERR_INVALID, "NULL spec, widths or needed");
  }
  return plan_create(out, 1, &spec, nullptr, nullptr, false, d_in, n_layers, widths, n_needed, needed, prec,
                     mem_budget_bytes, flags);
}

jet_status jet_plan_create_loss(jet_plan_t* out, int32_t n_terms, const jet_loss_term* terms, int32_t d_in,
                                int32_t n_layers, const int32_t* widths, int32_t n_needed, const jet_chan* needed,
                                jet_precision prec, size_t mem_budget_bytes, int32_t flags) {
  if (out) *out = nullptr;
  if (!terms || n_terms < 1 || n_terms > kMaxGroups)
    return fail(JET_ERR_INVALID, "a composite loss takes 1..%d terms", kMaxGroups);
  std::vector<const jet_residual_spec*> specs(n_terms);
  std::vector<double> weights(n_terms);
  std::vector<int32_t> paired(n_terms);
  for (int g = 0; g < n_terms; ++g) {
    specs[g] = terms[g].spec;
    weights[g] = terms[g].weight;
    paired[g] = terms[g].paired ? 1 : 0;
    if (!(terms[g].weight >= 0.0)) return fail(JET_ERR_INVALID, "loss term %d: weight must be >= 0", g);
  }
  return plan_create(out, n_terms, specs.data(), weights.data(), paired.data(), true, d_in, n_layers, widths,
                     n_needed, needed, prec, mem_budget_bytes, flags);
}

jet_status jet_plan_set_term_points(jet_plan_t p, const int64_t* counts) {
  if (!p || !counts) return fail(JET_ERR_INVALID, "NULL plan or counts");
  if (p->n_groups == 0) return fail(JET_ERR_INVALID, "the plan has one residual over all points (no loss terms)");
  long long start = 0;
  for (int g = 0; g < p->n_groups; ++g) {
    if (counts[g] < 0) return fail(JET_ERR_INVALID, "loss term %d: negative point count", g);
    if (p->groups[g].paired && ((start | counts[g]) & 1))
      return fail(JET_ERR_INVALID, "paired loss term %d must start at an even point index and hold whole pairs", g);
    start += counts[g];
  }
  p->group_counts.assign(counts, counts + p->n_groups);
  return JET_OK;
}

jet_status jet_plan_get_info(jet_plan_t p, jet_plan_info* info) {
  if (!p || !info) return fail(JET_ERR_INVALID, "NULL plan or info");
  memset(info, 0, sizeof(*info));
  info->d_in = p->d;
  info->n_out = p->n_out;
  info->n_layers = p->L;
  info->n_channels = p->C;
  info->closure_class = p->cls;
  snprintf(info->class_name, sizeof(info->class_name), "%s", kClassInfo[p->cls].name);
  info->n_params = p->n_params;
  info->precision = p->prec;
  info->store_mode = p->store != nullptr;
  info->store_max_points = p->store_max_points;
  info->tile_points = p->tc ? tc_tile_points(p->tcp) : p->P;
  info->grid_ctas = p->tc ? tc_grid(p->tcp) : p->grid;
  info->workspace_bytes = p->tc ? tc_workspace_bytes(p->tcp) : p->ws_bytes;
  info->ctas_per_sm = p->tc ? tc_ctas_per_sm(p->tcp) : p->ctas_per_sm;
  info->cta_threads = p->tc ? tc_threads(p->tcp) : kSimtThreads;
  info->wgrad_chunk_fp32 = p->tc ? tc_wgrad_chunk_fp32(p->tcp) : (p->wacc_off >= 0 ? 1 : 0);
  return JET_OK;
}

jet_status jet_plan_profile(jet_plan_t p, int32_t enable) {
  if (!p) return fail(JET_ERR_INVALID, "NULL plan");
  p->profiling = enable != 0;
  return JET_OK;
}

jet_status jet_plan_profile_read(jet_plan_t p, int64_t* launches, double* total_ms) {
  if (!p || !launches || !total_ms) return fail(JET_ERR_INVALID, "NULL argument");
  double tot = 0.0;
  for (auto& e : p->prof) {
    cudaError_t err = cudaEventSynchronize(e.second);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e.first, e.second);
    if (err != cudaSuccess) return cuda_fail(err, "profile events");
    tot += ms;
  }
  *launches = (int64_t)p->prof.size();
  *total_ms = tot;
  for (auto& e : p->prof) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  p->prof.clear();
  return JET_OK;
}

jet_status jet_plan_destroy(jet_plan_t p) {
  if (!p) return JET_OK;
  free_plan_ws(p);
  delete p;
  return JET_OK;
}

}  // extern "C"

namespace {

// Fill the per-call instance descriptor of the SIMT kernel.
void fill_instance(const jet_plan_s* p, const void* params, const void* X, long long N, const void* source,
                   void* r_out, int max_chunks, DevInstance& I) {
  memset(&I, 0, sizeof(I));
  I.L = p->L;
  I.d = p->d;
  I.n_out = p->n_out;
  I.n_res = p->n_res;
  for (int l = 0; l <= p->L; ++l) I.widths[l] = p->widths[l];
  for (int l = 0; l < p->L; ++l) {
    I.off_W[l] = p->off_W[l];
    I.off_b[l] = p->off_b[l];
  }
  I.n_params = p->n_params;
  I.params = params;
  I.Wt = p->Wt;
  I.X = X;
  I.source = source;
  I.r_out = r_out;
  I.N = N;
  I.inv_N = N > 0 ? 1.0 / (double)N : 0.0;
  I.n_terms = (int)p->terms.size();
  for (int m = 0; m < I.n_terms; ++m) I.terms[m] = p->terms[m];
  if (p->n_groups > 0) {
    I.inv_N = 1.0;  // each term's mean is in its scale
    I.n_groups = fill_groups(p, I.groups);
  }
  I.P = p->P;
  I.pitch = p->pitch;
  I.S = p->S;
  I.n_tiles = (N + p->P - 1) / p->P;
  long long chunks = std::min<long long>(std::max<long long>(I.n_tiles, 1), max_chunks);
  I.tiles_per_chunk = (int)((I.n_tiles + chunks - 1) / chunks);
  if (I.tiles_per_chunk < 1) I.tiles_per_chunk = 1;
  I.n_chunks = (int)((I.n_tiles + I.tiles_per_chunk - 1) / I.tiles_per_chunk);
  I.chunk_base = 0;
  I.grad_slices = p->grad_slices;
  I.loss_slices = p->loss_slices;
  I.store = nullptr;
  I.store_tile_stride = p->store_tile_stride;
  I.wacc_off = p->wacc_off;
}

jet_status check_call(const jet_plan_s* p, const void* params, const void* X, long long N, const void* source) {
  if (!p) return fail(JET_ERR_INVALID, "NULL plan");
  if (N < 0) return fail(JET_ERR_INVALID, "N < 0");
  if (p->n_groups > 0) {
    if ((int)p->group_counts.size() != p->n_groups)
      return fail(JET_ERR_INVALID, "a composite-loss plan needs jet_plan_set_term_points before its calls");
    long long tot = 0;
    for (long long c : p->group_counts) tot += c;
    if (tot != N) return fail(JET_ERR_INVALID, "N (%lld) differs from the loss terms' points (%lld)", N, tot);
  }
  if (!params) return fail(JET_ERR_INVALID, "NULL params");
  if (N > 0 && !X) return fail(JET_ERR_INVALID, "NULL X");
  if (p->has_source && N > 0 && !source) return fail(JET_ERR_INVALID, "the residual has a source: pass it");
  if (!p->has_source && source) return fail(JET_ERR_INVALID, "the residual has no source term");
  return JET_OK;
}

jet_status run_simt(jet_plan_s* p, int mode, const DevInstance& I, cudaStream_t s) {
  SimtArgs a;
  memset(&a, 0, sizeof(a));
  a.mode = mode;
  a.n_inst = 1;
  a.insts = nullptr;
  a.inst0 = I;
  a.n_items = I.n_chunks;
  a.item_inst = nullptr;
  a.scratch = p->scratch;
  a.scratch_stride = p->scratch_stride;
  int grid = std::min(p->grid, I.n_chunks);
  ProfScope prof(p, s);
  CK(simt_launch(p->cls, p->fp64, a, grid, p->smem, s));
  return JET_OK;
}

ReduceJob make_job(const DevInstance& I, void* grad_out, double* loss_out, bool with_grad) {
  ReduceJob j;
  memset(&j, 0, sizeof(j));
  j.grad_slices = I.grad_slices;
  j.loss_slices = I.loss_slices;
  j.n_chunks = I.n_chunks;
  j.n_params = with_grad ? I.n_params : 0;
  j.inv_N = I.inv_N;
  j.grad_out = grad_out;
  j.loss_out = loss_out;
  return j;
}

}  // namespace

extern "C" {

jet_status jet_forward_residual(jet_plan_t p, const void* params, const void* X, int64_t N, const void* source,
                                void* r_out, double* loss_out, jet_stream_t stream) {
  jet_status st = check_call(p, params, X, N, source);
  if (st != JET_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (p->tc) return tc_forward(p, p->tcp, params, X, N, source, r_out, loss_out, s);
  if (N == 0) {
    if (loss_out) CK(cudaMemsetAsync(loss_out, 0, sizeof(double), s));
    return JET_OK;
  }
  DevInstance I;
  fill_instance(p, params, X, N, source, r_out, p->grid, I);
  const bool store = p->store && N <= p->store_max_points;
  if (store) I.store = p->store;
  CK(launch_transpose_weights(I, p->fp64, p->Wt, s));
  st = run_simt(p, MODE_FWD, I, s);
  if (st != JET_OK) return st;
  ReduceJob j = make_job(I, nullptr, loss_out, false);
  if (loss_out) CK(launch_reduce(nullptr, j, 1, 1, p->fp64, false, 1, 0.f, s));
  p->st_valid = store;
  p->st_params = params;
  p->st_X = X;
  p->st_src = source;
  p->st_N = N;
  return JET_OK;
}

jet_status jet_backward_params(jet_plan_t p, const void* params, const void* X, int64_t N, const void* source,
                               void* grad_out, void* r_out, double* loss_out, jet_stream_t stream) {
  jet_status st = check_call(p, params, X, N, source);
  if (st != JET_OK) return st;
  if (!grad_out) return fail(JET_ERR_INVALID, "NULL grad_out");
  cudaStream_t s = (cudaStream_t)stream;
  if (p->tc) return tc_backward(p, p->tcp, params, X, N, source, grad_out, r_out, loss_out, s);
  if (N == 0) {
    CK(cudaMemsetAsync(grad_out, 0, p->n_params * p->elem, s));
    if (loss_out) CK(cudaMemsetAsync(loss_out, 0, sizeof(double), s));
    return JET_OK;
  }
  DevInstance I;
  fill_instance(p, params, X, N, source, r_out, p->grid, I);
  const bool from_store = p->st_valid && p->st_params == params && p->st_X == X && p->st_N == N &&
                          p->st_src == source;
  if (from_store) I.store = p->store;
  CK(launch_transpose_weights(I, p->fp64, p->Wt, s));
  st = run_simt(p, from_store ? MODE_BWD_STORE : MODE_FWD_BWD, I, s);
  if (st != JET_OK) return st;
  ReduceJob j = make_job(I, grad_out, loss_out, true);
  CK(launch_reduce(nullptr, j, 1, I.n_params, p->fp64, false, 1, 0.f, s));
  return JET_OK;
}

}  // extern "C"

// Adam step t = `step`, or *step_ctr + 1 (then incremented) with a device counter
static jet_status train_step(jet_plan_t p, void* params, void* adam_m, void* adam_v, int64_t step,
                             long long* step_ctr, float lr, const void* X, int64_t N, const void* source,
                             double* loss_out, cudaStream_t s) {
  jet_status st = check_call(p, params, X, N, source);
  if (st != JET_OK) return st;
  if (!adam_m || !adam_v) return fail(JET_ERR_INVALID, "NULL Adam state");
  if (N < 1) return fail(JET_ERR_INVALID, "train step needs N >= 1");
  p->st_valid = false;  // params change in place
  if (p->tc) return tc_train_step(p, p->tcp, params, adam_m, adam_v, step, step_ctr, lr, X, N, source, loss_out, s);
  DevInstance I;
  fill_instance(p, params, X, N, source, nullptr, p->grid, I);
  CK(launch_transpose_weights(I, p->fp64, p->Wt, s));
  st = run_simt(p, MODE_FWD_BWD, I, s);
  if (st != JET_OK) return st;
  ReduceJob j = make_job(I, nullptr, loss_out, true);
  j.params = params;
  j.m = adam_m;
  j.v = adam_v;
  CK(launch_reduce(nullptr, j, 1, I.n_params, p->fp64, true, step, lr, s, step_ctr));
  return JET_OK;
}

extern "C" {

jet_status jet_train_step(jet_plan_t p, void* params, void* adam_m, void* adam_v, int64_t step, float lr,
                          const void* X, int64_t N, const void* source, double* loss_out, jet_stream_t stream) {
  if (step < 1) return fail(JET_ERR_INVALID, "step must be >= 1");
  return train_step(p, params, adam_m, adam_v, step, nullptr, lr, X, N, source, loss_out, (cudaStream_t)stream);
}

jet_status jet_train_step_dev(jet_plan_t p, void* params, void* adam_m, void* adam_v, int64_t* step_counter,
                              float lr, const void* X, int64_t N, const void* source, double* loss_out,
                              jet_stream_t stream) {
  if (!step_counter) return fail(JET_ERR_INVALID, "NULL step counter");
  return train_step(p, params, adam_m, adam_v, 1, reinterpret_cast<long long*>(step_counter), lr, X, N, source,
                    loss_out, (cudaStream_t)stream);
}

jet_status jet_debug_activation(jet_plan_t p, int32_t kind, int64_t n, const double* z, const double* v, double* out,
                                jet_stream_t stream) {
  if (!p || !z || !out || (kind != 0 && !v)) return fail(JET_ERR_INVALID, "NULL argument");
  if (kind < 0 || kind > 2) return fail(JET_ERR_INVALID, "kind must be 0, 1 or 2");
  CK(debug_act(p->cls, kind, n, z, v, out, (cudaStream_t)stream));
  return JET_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches

struct jet_batch_s {
  std::vector<jet_plan_t> plans;
  int cls = -1;
  bool fp64 = false;
  bool tc = false;
  int grid = 0;
  size_t smem = 0;
  int max_chunks_per_inst = 16;
  // device workspace
  DevInstance* d_insts = nullptr;
  int* d_item_inst = nullptr;
  int* d_next = nullptr;  // the kernel's item counter
  ReduceJob* d_jobs = nullptr;
  double* grad_slices = nullptr;
  double* loss_slices = nullptr;
  void* Wt = nullptr;
  void* scratch = nullptr;
  long long scratch_stride = 0;
  std::vector<long long> slice_off, wt_off;
  // pinned host staging for the per-call descriptors
  DevInstance* h_insts = nullptr;
  int* h_item_inst = nullptr;
  ReduceJob* h_jobs = nullptr;
  int max_items = 0;
  TcBatch* tcb = nullptr;
  // the pinned staging buffers are rewritten by the next call only after the
  // uploads of this one have read them
  cudaEvent_t copied = nullptr;
  bool have_prev = false;
};

namespace {

void free_batch(jet_batch_s* b) {
  cudaFree(b->d_insts);
  cudaFree(b->d_item_inst);
  cudaFree(b->d_next);
  cudaFree(b->d_jobs);
  cudaFree(b->grad_slices);
  cudaFree(b->loss_slices);
  cudaFree(b->Wt);
  cudaFree(b->scratch);
  cudaFreeHost(b->h_insts);
  cudaFreeHost(b->h_item_inst);
  cudaFreeHost(b->h_jobs);
  if (b->tcb) tc_batch_destroy(b->tcb);
  if (b->copied) cudaEventDestroy(b->copied);
}

// Build the per-call work list: every instance is split into chunks of point
// tiles; items are ordered by estimated cost, largest first, and pulled by the
// persistent CTAs in that order.
jet_status batch_prepare(jet_batch_s* b, const void* const* params, const void* const* X, const int64_t* N,
                         const void* const* source, void* const* r_out, int* n_items_out, cudaStream_t s) {
  const int n = (int)b->plans.size();
  long long total_tiles = 0;
  for (int i = 0; i < n; ++i) {
    jet_status st = check_call(b->plans[i], params[i], X[i], N[i], source ? source[i] : nullptr);
    if (st != JET_OK) return st;
    total_tiles += (N[i] + b->plans[i]->P - 1) / b->plans[i]->P;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (b->have_prev && cs == cudaStreamCaptureStatusNone) cudaEventSynchronize(b->copied);
  // target about four items per CTA
  long long target_tiles = std::max<long long>(1, (total_tiles + 4LL * b->grid - 1) / (4LL * b->grid));
  std::vector<std::pair<double, int>> cost;  // (cost, item) for ordering
  std::vector<int> item_inst;
  int chunk_base = 0;
  for (int i = 0; i < n; ++i) {
    jet_plan_s* p = b->plans[i];
    DevInstance& I = b->h_insts[i];
    const long long tiles = (N[i] + p->P - 1) / p->P;
    long long want = std::min<long long>(b->max_chunks_per_inst, std::max<long long>(1, (tiles + target_tiles - 1) / target_tiles));
    fill_instance(p, params[i], X[i], N[i], source ? source[i] : nullptr, r_out ? r_out[i] : nullptr, (int)want, I);
    I.Wt = (char*)b->Wt + b->wt_off[i] * p->elem;
    I.grad_slices = b->grad_slices + b->slice_off[i];
    I.loss_slices = b->loss_slices + (long long)i * b->max_chunks_per_inst;
    I.chunk_base = chunk_base;
    double per_tile = 0;
    for (int l = 2; l < p->L; ++l) per_tile += (double)p->widths[l - 1] * p->widths[l];
    per_tile = (per_tile + 64.0) * p->C * p->P;
    for (int c = 0; c < I.n_chunks; ++c) {
      const long long t0 = (long long)c * I.tiles_per_chunk;
      const long long nt = std::min<long long>(tiles, t0 + I.tiles_per_chunk) - t0;
      cost.push_back({per_tile * (double)nt, chunk_base + c});
      item_inst.push_back(i);
    }
    chunk_base += I.n_chunks;
  }
  if (chunk_base > b->max_items) return fail(JET_ERR_INVALID, "internal: work list overflow");
  std::vector<int> order(chunk_base);
  for (int k = 0; k < chunk_base; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x].first > cost[y].first; });
  // the kernel walks items in list order; item ids keep their instance chunk
  // numbering through chunk_base, so list position k maps to item order[k]
  for (int k = 0; k < chunk_base; ++k) b->h_item_inst[k] = order[k];
  // h_item_inst[k] holds the global item id; instance lookup table follows it
  for (int k = 0; k < chunk_base; ++k) b->h_item_inst[chunk_base + k] = item_inst[k];
  CK(cudaMemcpyAsync(b->d_insts, b->h_insts, sizeof(DevInstance) * n, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(b->d_item_inst, b->h_item_inst, sizeof(int) * 2 * chunk_base, cudaMemcpyHostToDevice, s));
  *n_items_out = chunk_base;
  return JET_OK;
}

}  // namespace

extern "C" {

jet_status jet_batch_create(jet_batch_t* out, int32_t n, const jet_plan_t* plans, int32_t flags) {
  (void)flags;
  if (!out || n < 1 || !plans) return fail(JET_ERR_INVALID, "bad batch arguments");
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (!plans[i]) return fail(JET_ERR_INVALID, "plan %d is NULL", i);
  const bool tc = plans[0]->tc;
  for (int i = 1; i < n; ++i) {
    if (plans[i]->tc != tc || plans[i]->fp64 != plans[0]->fp64)
      return fail(JET_ERR_UNSUPPORTED, "batch plans must share the precision family");
    if (plans[i]->cls != plans[0]->cls) return fail(JET_ERR_UNSUPPORTED, "batch plans must share the channel set");
  }
  jet_batch_s* b = new jet_batch_s();
  b->plans.assign(plans, plans + n);
  b->cls = plans[0]->cls;
  b->fp64 = plans[0]->fp64;
  b->tc = tc;
  if (tc) {
    jet_status st = tc_batch_create(b->plans, &b->tcb);
    if (st != JET_OK) {
      delete b;
      return st;
    }
    *out = b;
    return JET_OK;
  }
  size_t smem = 0;
  long long scr = 0, slices = 0, wt = 0;
  for (int i = 0; i < n; ++i) {
    smem = std::max(smem, plans[i]->smem);
    scr = std::max(scr, plans[i]->scratch_stride);
    b->slice_off.push_back(slices);
    slices += (long long)b->max_chunks_per_inst * plans[i]->n_params;
    b->wt_off.push_back(wt);
    wt += weight_ws_elems(plans[i]->n_params);
  }
  b->smem = smem;
  int per_sm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, dev);
  if (e == cudaSuccess) e = simt_occupancy(b->cls, b->fp64, smem, &per_sm);
  if (e != cudaSuccess || per_sm < 1) {
    delete b;
    return e != cudaSuccess ? cuda_fail(e, "batch occupancy") : fail(JET_ERR_UNSUPPORTED, "batch tile does not fit");
  }
  b->grid = prop.multiProcessorCount * per_sm;
  b->scratch_stride = scr;
  b->max_items = n * b->max_chunks_per_inst;
  const size_t elem = b->fp64 ? 8 : 4;
  e = cudaMalloc((void**)&b->d_insts, sizeof(DevInstance) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_item_inst, sizeof(int) * 2 * b->max_items);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_next, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_jobs, sizeof(ReduceJob) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->grad_slices, sizeof(double) * std::max<long long>(slices, 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->loss_slices, sizeof(double) * b->max_items);
  if (e == cudaSuccess) e = cudaMalloc(&b->Wt, elem * std::max<long long>(wt, 1));
  if (e == cudaSuccess) e = cudaMalloc(&b->scratch, elem * (size_t)b->grid * std::max<long long>(scr, 1));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_insts, sizeof(DevInstance) * n);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_item_inst, sizeof(int) * 2 * b->max_items);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_jobs, sizeof(ReduceJob) * n);
  if (e != cudaSuccess) {
    free_batch(b);
    delete b;
    return cuda_fail(e, "batch workspace");
  }
  *out = b;
  return JET_OK;
}

static jet_status batch_run(jet_batch_t b, const void* const* params, void* const* adam_m, void* const* adam_v,
                            int64_t step, long long* step_ctr, float lr, const void* const* X, const int64_t* N,
                            const void* const* source, void* const* grad_out, double* loss_out, bool adam,
                            cudaStream_t s) {
  const int n = (int)b->plans.size();
  int n_items = 0;
  jet_status st = batch_prepare(b, params, X, N, source, nullptr, &n_items, s);
  if (st != JET_OK) return st;
  for (int i = 0; i < n; ++i) CK(launch_transpose_weights(b->h_insts[i], b->fp64, (void*)b->h_insts[i].Wt, s));
  SimtArgs a;
  memset(&a, 0, sizeof(a));
  a.mode = MODE_FWD_BWD;
  a.n_inst = n;
  a.insts = b->d_insts;
  a.n_items = n_items;
  a.item_inst = b->d_item_inst;
  a.scratch = b->scratch;
  a.scratch_stride = b->scratch_stride;
  a.item_next = b->d_next;
  CK(cudaMemsetAsync(b->d_next, 0, sizeof(int), s));
  CK(simt_launch(b->cls, b->fp64, a, std::min(b->grid, n_items), b->smem, s));
  long long maxp = 0;
  for (int i = 0; i < n; ++i) {
    ReduceJob j = make_job(b->h_insts[i], adam ? nullptr : grad_out[i], loss_out ? loss_out + i : nullptr, true);
    if (adam) {
      j.params = (void*)params[i];
      j.m = adam_m[i];
      j.v = adam_v[i];
    }
    b->h_jobs[i] = j;
    maxp = std::max(maxp, j.n_params);
  }
  CK(cudaMemcpyAsync(b->d_jobs, b->h_jobs, sizeof(ReduceJob) * n, cudaMemcpyHostToDevice, s));
  if (!b->copied) CK(cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming));
  cudaStreamCaptureStatus cs2 = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs2);
  if (cs2 == cudaStreamCaptureStatusNone) {  // a captured upload replays from the staging of the latest call
    CK(cudaEventRecord(b->copied, s));
    b->have_prev = true;
  }
  CK(launch_reduce(b->d_jobs, b->h_jobs[0], n, maxp, b->fp64, adam, step, lr, s, step_ctr));
  return JET_OK;
}

jet_status jet_batch_backward(jet_batch_t b, const void* const* params, const void* const* X, const int64_t* N,
                              const void* const* source, void* const* grad_out, double* loss_out,
                              jet_stream_t stream) {
  if (!b || !params || !X || !N || !grad_out) return fail(JET_ERR_INVALID, "NULL batch argument");
  if (b->tc) return tc_batch_run(b->tcb, b->plans, params, nullptr, nullptr, 0, nullptr, 0.f, X, N, source,
                                 grad_out, loss_out, false, (cudaStream_t)stream);
  return batch_run(b, params, nullptr, nullptr, 0, nullptr, 0.f, X, N, source, grad_out, loss_out, false,
                   (cudaStream_t)stream);
}

static jet_status batch_train(jet_batch_t b, void* const* params, void* const* adam_m, void* const* adam_v,
                              int64_t step, long long* step_ctr, float lr, const void* const* X, const int64_t* N,
                              const void* const* source, double* loss_out, cudaStream_t s) {
  if (!b || !params || !adam_m || !adam_v || !X || !N) return fail(JET_ERR_INVALID, "NULL batch argument");
  if (b->tc) return tc_batch_run(b->tcb, b->plans, (const void* const*)params, adam_m, adam_v, step, step_ctr, lr,
                                 X, N, source, nullptr, loss_out, true, s);
  return batch_run(b, (const void* const*)params, adam_m, adam_v, step, step_ctr, lr, X, N, source, nullptr,
                   loss_out, true, s);
}

jet_status jet_batch_train_step(jet_batch_t b, void* const* params, void* const* adam_m, void* const* adam_v,
                                int64_t step, float lr, const void* const* X, const int64_t* N,
                                const void* const* source, double* loss_out, jet_stream_t stream) {
  if (step < 1) return fail(JET_ERR_INVALID, "step must be >= 1");
  return batch_train(b, params, adam_m, adam_v, step, nullptr, lr, X, N, source, loss_out, (cudaStream_t)stream);
}

jet_status jet_batch_train_step_dev(jet_batch_t b, void* const* params, void* const* adam_m, void* const* adam_v,
                                    int64_t* step_counter, float lr, const void* const* X, const int64_t* N,
                                    const void* const* source, double* loss_out, jet_stream_t stream) {
  if (!step_counter) return fail(JET_ERR_INVALID, "NULL step counter");
  return batch_train(b, params, adam_m, adam_v, 1, reinterpret_cast<long long*>(step_counter), lr, X, N, source,
                     loss_out, (cudaStream_t)stream);
}

jet_status jet_batch_destroy(jet_batch_t b) {
  if (!b) return JET_OK;
  free_batch(b);
  delete b;
  return JET_OK;
}

}  // extern "C"
