// Residual stage of a composite loss (Sec. 3.1.1, all-points batching): the
// network's output jets of a tile's points are split among the loss terms by
// point index, each term assembles its own residual, and the loss adds
// scale_g * r^2 per residual.  Shared by the SIMT and tensor-core kernels,
// whose output jets sit in UO[(o * C + channel) * P + n] and whose residual
// adjoints go to UB in the same layout.
#pragma once

#include "jet_internal.h"

namespace jet {

// Per-point loop: thread of point n assembles the residual of n's term at n
// (and, for a paired term, reads the pair's second point n + 1, which lies in
// the same tile because terms start at even indices and tiles hold an even
// number of points); it writes r_out, adds the loss and, in the backward pass,
// the adjoints dL/du of both points.  No other thread touches those UB
// entries, so the adds need no atomics.  UB must be zeroed before (bwd).
template <class T>
__device__ double grouped_residual(const DevTerm* terms, const DevGroup* groups, int n_groups, int n_res_max,
                                   const T* UO, T* UB, int P, long long n0, int nvalid, const T* src, T* rout,
                                   bool bwd, int tid, int nthr) {
  double loss = 0.0;
  for (int n = tid; n < nvalid; n += nthr) {
    const long long gn = n0 + n;
    int g = 0;
    while (g + 1 < n_groups && gn >= groups[g + 1].start) ++g;
    const DevGroup& G = groups[g];
    if (G.paired && ((gn - G.start) & 1)) continue;  // second point of a pair: its first point's thread
    T r[kMaxRes];
#pragma unroll
    for (int c = 0; c < kMaxRes; ++c) r[c] = (c < G.n_res && G.has_source && src) ? -src[gn * n_res_max + c] : T(0);
    for (int m = G.t0; m < G.t1; ++m) {
      const DevTerm& tm = terms[m];
      T prod = T(tm.coef);
      for (int f = 0; f < tm.nfac; ++f) prod *= UO[tm.fac[f] * P + n + ((tm.pmask >> f) & 1)];
#pragma unroll
      for (int c = 0; c < kMaxRes; ++c)
        if (c == tm.comp) r[c] += prod;
    }
    if (rout)
      for (int c = 0; c < n_res_max; ++c) {
        rout[gn * n_res_max + c] = c < G.n_res ? r[c] : T(0);
        if (G.paired) rout[(gn + 1) * n_res_max + c] = T(0);
      }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kMaxRes; ++c) s += (double)r[c] * (double)r[c];
    loss += G.scale * s;
    if (!bwd) continue;
    const T two_scale = T(2.0 * G.scale);
    for (int m = G.t0; m < G.t1; ++m) {
      const DevTerm& tm = terms[m];
      T rc = T(0);
#pragma unroll
      for (int c = 0; c < kMaxRes; ++c)
        if (c == tm.comp) rc = r[c];
      const T gg = two_scale * rc * T(tm.coef);
      for (int f = 0; f < tm.nfac; ++f) {
        T prod = gg;
        for (int h = 0; h < tm.nfac; ++h)
          if (h != f) prod *= UO[tm.fac[h] * P + n + ((tm.pmask >> h) & 1)];
        UB[tm.fac[f] * P + n + ((tm.pmask >> f) & 1)] += prod;
      }
    }
  }
  return loss;
}

}  // namespace jet
