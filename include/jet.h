/*
 * jet.h -- C ABI of libjet: residual-specific partial-jet PINN kernels for
 * NVIDIA GB300 (sm_103a).
 *
 * What the library computes (Sec. 2.2 of "Verified residual-specific explicit
 * derivative kernels for physics-informed learning and discretized PDE
 * adjoints"):
 *
 *   * a tanh multilayer perceptron u_theta: R^d -> R^n_out (Eq. 1:
 *     z^l = W^l a^{l-1} + b^l, a^l = tanh(z^l) for the hidden layers, linear
 *     output layer);
 *   * the coordinate derivatives d^alpha u_theta that a PDE residual needs,
 *     propagated layer by layer as a *partial jet*: only the multi-indices of
 *     the residual plus their lower-order chain are carried (Sec. 2.2,
 *     "on-demand partial-jet strategy"); every layer applies W^l to all jet
 *     channels at once with the bias on the value channel only (Eq. 2-3 and
 *     the "fused GEMM" of Sec. 2.2), and the tanh composes the jet in closed
 *     form (Eq. 2, Eq. 3 and their higher-order recursion);
 *   * the residual r_theta(x) = N(u, d_i u, d_ij u, ...) (Sec. 2.2), here a
 *     sum of monomials of output-jet entries minus an optional source;
 *   * the loss L = sum_c (1/N) sum_n r_{c,n}^2 and its gradient with respect
 *     to every parameter (Sec. 3.1.1: reverse-mode differentiation of the
 *     scalar loss), by a hand-written reverse sweep of the jet program;
 *   * one full-batch Adam step (Sec. 3.1.1, learning rate 1e-3 in the paper).
 *
 * Conventions shared by every call:
 *   * All device pointers are CUDA device (or managed) memory owned by the
 *     caller; the library never frees them.  Calls are asynchronous on the
 *     given stream (0 = legacy default stream) unless stated.
 *   * Value type: a plan created with JET_FP64 takes and returns double for
 *     params, X, source, r_out and grad_out; every other precision takes and
 *     returns float.  Losses are always double.
 *   * Parameter packing: for l = 1..L, W^l row-major [out][in] followed by
 *     b^l [out] (Eq. 1 orientation), all layers back to back.
 *   * Points X: row-major [N][d]; source: row-major [N][n_res]; r_out:
 *     row-major [N][n_res].
 *   * Errors: every call returns a jet_status and never aborts; a thread-
 *     local message is available from jet_last_error().  Shape and spec
 *     errors are caught by jet_plan_create.
 *   * CUDA graphs: the compute calls of a plan or batch may be recorded by
 *     stream capture once the same call has run outside capture (which sizes
 *     any store and loads the kernels).  A call being captured allocates
 *     nothing and reads nothing back to the host; a bounded device wait that
 *     times out during a replay is reported by the next call made outside
 *     capture.  jet_train_step_dev keeps the Adam step on the device, so
 *     replays advance it.
 */
#ifndef JET_H_
#define JET_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct jet_plan_s* jet_plan_t;
typedef struct jet_batch_s* jet_batch_t;
typedef void* jet_stream_t; /* a cudaStream_t */

typedef enum {
  JET_OK = 0,
  JET_ERR_INVALID = 1,     /* bad argument, shape or spec */
  JET_ERR_NOT_CLOSED = 2,  /* needed multi-indices not downward closed */
  JET_ERR_UNSUPPORTED = 3, /* valid request outside what this build supports */
  JET_ERR_OOM = 4,         /* device allocation failed or budget too small */
  JET_ERR_CUDA = 5,        /* a CUDA runtime call or launch failed */
  JET_ERR_TIMEOUT = 6      /* a bounded device-side wait gave up */
} jet_status;

typedef enum {
  JET_FP64 = 0,     /* FP64 SIMT kernels */
  JET_FP32 = 1,     /* plain FP32 SIMT kernels (no tensor cores) */
  JET_TF32 = 2,     /* reserved: not provided by this build (jet_plan_create
                       returns JET_ERR_UNSUPPORTED) */
  JET_BF16 = 3,     /* tcgen05 kind::f16 (bf16) jet GEMMs, FP32 accumulation */
  JET_BF16X3 = 4    /* as JET_BF16, plus split bf16 hi/lo products on the
                       highest-order channels (hidden width <= 128) */
} jet_precision;

/* plan flags */
#define JET_FLAG_AUTO_CLOSE 0x1  /* close `needed` downward instead of failing */
#define JET_FLAG_STORE 0x2       /* FP64/FP32 forms: jet_forward_residual keeps
                                    the hidden z-jets (if they fit the budget)
                                    for the next jet_backward_params on the
                                    same inputs.  BF16 forms: the backward pass
                                    keeps every tile's layer inputs and adjoints
                                    in HBM (within the budget) and computes the
                                    weight gradients as one GEMM per layer */
/* Tile override (used by the autotuner): points per tile of the fused kernel,
 * P = 8 * JET_FLAG_TILE_GET(flags) when nonzero.  The plan rejects a P its
 * kernel cannot run (JET_ERR_UNSUPPORTED); 0 keeps the built-in choice. */
#define JET_FLAG_TILE(p8) (((p8)&0xff) << 8)
#define JET_FLAG_TILE_GET(flags) (((flags) >> 8) & 0xff)
/* CTA shape override of the tensor-core kernel (used by the autotuner):
 * n = 1 runs one CTA of 16 warps per SM, n = 2 two CTAs of 8 warps per SM
 * (each with its own tile, so one CTA's activation epilogue overlaps the
 * other's MMAs and copies).  0 keeps the built-in choice; a shape whose tile
 * does not fit shared memory or TMEM gives JET_ERR_UNSUPPORTED.  Ignored by
 * the FP64 and FP32 forms. */
#define JET_FLAG_CTAS(n) (((n)&0x3) << 16)
#define JET_FLAG_CTAS_GET(flags) (((flags) >> 16) & 0x3)

/* One derivative channel d^alpha u_out: alpha[i] = order in coordinate i. */
typedef struct {
  int32_t out;
  uint8_t alpha[4];
} jet_chan;

/* coef * prod_{j < n_fac} d^{fac[j].alpha} u_{fac[j].out} */
typedef struct {
  double coef;
  int32_t n_fac; /* 0..4 */
  jet_chan fac[4];
} jet_monomial;

/* r_c = sum_m mono[c][m] - source_c  for c < n_res. */
typedef struct {
  int32_t n_res;                   /* 1..4 */
  const int32_t* n_mono;           /* [n_res] */
  const jet_monomial* const* mono; /* [n_res][n_mono[c]] */
  int32_t has_source;              /* 1: calls pass source [N][n_res] */
} jet_residual_spec;

typedef struct {
  int32_t d_in, n_out, n_layers;
  int32_t n_channels;      /* C = 1 + k channels carried per unit */
  int32_t closure_class;   /* index of the compiled channel set used */
  char class_name[32];
  int64_t n_params;
  int32_t precision;
  int32_t store_mode;      /* 1 if jet_forward_residual stores z-jets */
  int64_t store_max_points;
  int32_t tile_points;     /* points per tile of the fused kernel */
  int32_t grid_ctas;       /* persistent CTAs per launch */
  size_t workspace_bytes;  /* device memory the plan owns */
  int32_t ctas_per_sm;     /* CTAs of the fused kernel resident per SM */
  int32_t cta_threads;     /* threads per CTA of the fused kernel */
  int32_t wgrad_chunk_fp32; /* 1: hidden-layer weight gradients computed per
                               tile add up in an FP32 accumulator per CTA and
                               reach the FP64 chunk sums once per chunk; 0:
                               they are added into the FP64 chunk sums per
                               tile (FP64 forms; FP32 plans whose FP64 chunk
                               sums fit in L2) */
} jet_plan_info;

/*
 * Create a plan for one PDE residual on one network shape.
 *   spec       residual (Sec. 2.2, r = N(u, du, ...)); copied.
 *   d_in       number of input coordinates (1..3).
 *   n_layers   number of weight layers L >= 2 (L-1 tanh hidden layers).
 *   widths     [L+1]: d_in, hidden widths..., n_out (n_out 1..4).  Hidden
 *              widths must be multiples of 4 and at most 256.
 *   needed     [n_needed] multi-indices the residual uses (the out field is
 *              ignored).  They must be downward closed (every alpha' <= alpha
 *              present, the value included) unless JET_FLAG_AUTO_CLOSE.  The
 *              plan carries the smallest compiled channel set containing them
 *              (Sec. 2.2: only the required states and their lower-order
 *              chain are propagated).
 *   prec       jet_precision.
 *   mem_budget_bytes  upper bound on plan-owned device memory for the store
 *              of JET_FLAG_STORE; 0 = no store.  Without a store the backward
 *              pass works in bounded memory by recomputing the jets of each
 *              tile from its layer inputs.  A BF16 store plan may pick a tile
 *              that fits shared memory only with the store (one activation
 *              buffer); its jet_backward_params / jet_train_step then return
 *              JET_ERR_OOM when N points do not fit the budget, and it cannot
 *              join a batch (JET_ERR_UNSUPPORTED).
 * On success *out owns device workspace until jet_plan_destroy.
 */
jet_status jet_plan_create(jet_plan_t* out, const jet_residual_spec* spec, int32_t d_in, int32_t n_layers,
                           const int32_t* widths, int32_t n_needed, const jet_chan* needed,
                           jet_precision prec, size_t mem_budget_bytes, int32_t flags);

/*
 * Composite PINN loss with all-points batching (Sec. 3.1.1): the training
 * loss of the paper's Burgers and lid-driven cavity cases sums weighted terms
 * -- initial-condition, boundary-condition and PDE-residual terms -- each
 * over its own point set, and the network (with its derivative channels) is
 * evaluated once on all points concatenated, the outputs split afterwards:
 *
 *   L = sum_g weight_g * (1 / M_g) * sum_{residuals m of term g} sum_c r_{g,c,m}^2
 *
 * Term g owns a contiguous block of the concatenated points, in term order
 * (counts from jet_plan_set_term_points).  A plain term has one residual per
 * point (M_g = its points).  A paired term owns its points as consecutive
 * pairs (a, b) and has one residual per pair (M_g = half its points), whose
 * monomial factors read the jets at a, or at b when their jet_chan.out
 * carries JET_PAIR_SECOND: e.g. the periodic boundary conditions
 * u(0, t) - u(1, t) and u_x(0, t) - u_x(1, t).  A paired term must start at
 * an even point index.
 */
#define JET_PAIR_SECOND 0x100 /* jet_chan.out flag: factor read at the pair's second point */

typedef struct {
  const jet_residual_spec* spec; /* the term's residual (its own source flag) */
  double weight;                 /* weight_g >= 0 */
  int32_t paired;                /* 1: one residual per consecutive pair of points */
} jet_loss_term;

/*
 * Create a plan for a composite loss of n_terms (1..4) terms on one network
 * shape.  The carried channel set is the closure of `needed`, which must
 * cover every term's multi-indices (JET_FLAG_AUTO_CLOSE closes it); all other
 * arguments as jet_plan_create.  The plan's n_res is the largest of the
 * terms'.  Before its compute calls, jet_plan_set_term_points gives the point
 * count of every term; then every call takes X = the terms' points
 * concatenated in term order with N = their sum, source [N][n_res] (rows of
 * terms whose spec has no source are ignored) if any term has one, and
 * writes r_out [N][n_res] with each term's components at its residual points
 * (zeros at the second points of pairs and in components a term lacks).
 * loss_out is L above.  Batches accept such plans.
 */
jet_status jet_plan_create_loss(jet_plan_t* out, int32_t n_terms, const jet_loss_term* terms, int32_t d_in,
                                int32_t n_layers, const int32_t* widths, int32_t n_needed, const jet_chan* needed,
                                jet_precision prec, size_t mem_budget_bytes, int32_t flags);

/*
 * Point counts of a composite-loss plan's terms (host array [n_terms]) for
 * its next calls.  JET_ERR_INVALID for a plan with one residual, a negative
 * count, or a paired term that would not start at an even point index or
 * holds an odd number of points.  Host-side state only: a call captured in a
 * CUDA graph keeps the counts it was captured with.
 */
jet_status jet_plan_set_term_points(jet_plan_t plan, const int64_t* counts);

jet_status jet_plan_get_info(jet_plan_t plan, jet_plan_info* info);

/*
 * Residual and loss (Sec. 2.2 forward partial-jet pass, Eq. 1-3).
 *   params    device, packed (see top); X device [N][d]; source device
 *             [N][n_res] or NULL when the spec has none.
 *   r_out     device [N][n_res] or NULL.
 *   loss_out  device double scalar or NULL: sum_c (1/N) sum_n r_{c,n}^2.
 * N may be 0 (loss 0, nothing written to r_out).
 */
jet_status jet_forward_residual(jet_plan_t plan, const void* params, const void* X, int64_t N,
                                const void* source, void* r_out, double* loss_out, jet_stream_t stream);

/*
 * Gradient of the loss with respect to every parameter (Sec. 3.1.1 reverse
 * mode of the scalar loss, here a hand-written adjoint of the jet program).
 *   grad_out  device, packed like params (value type of the plan).
 *   loss_out  device double or NULL.
 *   r_out     device [N][n_res] or NULL (the residual of the same pass).
 * The hidden jets are recomputed tile by tile from the inputs, unless the plan
 * stores them and the previous jet_forward_residual on this plan used the same
 * params, X, N and source pointers (the caller must not have changed their
 * contents in between).
 */
jet_status jet_backward_params(jet_plan_t plan, const void* params, const void* X, int64_t N,
                               const void* source, void* grad_out, void* r_out, double* loss_out,
                               jet_stream_t stream);

/*
 * One full-batch Adam step on params in place (Sec. 3.1.1; beta1 0.9,
 * beta2 0.999, eps 1e-8, bias-corrected with the 1-based `step`).
 *   adam_m, adam_v  device, packed like params, value type of the plan;
 *                   zero before step 1.
 *   loss_out        device double or NULL: the loss BEFORE the update.
 * Works for every plan precision; the update runs in the parameters' value
 * type (FP64 for JET_FP64, FP32 otherwise).  `step` is a host value: a CUDA
 * graph that captures this call repeats that step's bias correction on every
 * replay.  Use jet_train_step_dev for replayed training loops.
 */
jet_status jet_train_step(jet_plan_t plan, void* params, void* adam_m, void* adam_v, int64_t step, float lr,
                          const void* X, int64_t N, const void* source, double* loss_out, jet_stream_t stream);

/*
 * jet_train_step with the Adam step counter in device memory (Sec. 3.1.1,
 * full-batch Adam).
 *   step_counter  device int64: the number of Adam steps already taken
 *                 (0 before the first).  The call performs step
 *                 t = *step_counter + 1 (bias corrections 1 - beta^t computed
 *                 on the device) and then increments *step_counter on the
 *                 stream, so k launches of the same captured CUDA graph take
 *                 k consecutive Adam steps.
 * Everything else as jet_train_step; both calls give identical results for
 * the same step number.
 */
jet_status jet_train_step_dev(jet_plan_t plan, void* params, void* adam_m, void* adam_v, int64_t* step_counter,
                              float lr, const void* X, int64_t N, const void* source, double* loss_out,
                              jet_stream_t stream);

jet_status jet_plan_destroy(jet_plan_t plan);

/*
 * Batched ensemble: n independent plans (same precision; any shapes and
 * residuals) run as ONE persistent launch over a work list of
 * (instance, chunk of point tiles) items.  Arrays are host arrays of n
 * device pointers / sizes.
 */
jet_status jet_batch_create(jet_batch_t* out, int32_t n, const jet_plan_t* plans, int32_t flags);
jet_status jet_batch_backward(jet_batch_t batch, const void* const* params, const void* const* X,
                              const int64_t* N, const void* const* source, void* const* grad_out,
                              double* loss_out /* device [n] or NULL */, jet_stream_t stream);
jet_status jet_batch_train_step(jet_batch_t batch, void* const* params, void* const* adam_m,
                                void* const* adam_v, int64_t step, float lr, const void* const* X,
                                const int64_t* N, const void* const* source,
                                double* loss_out /* device [n] or NULL */, jet_stream_t stream);
/* As jet_batch_train_step, with one device step counter shared by every
 * instance (see jet_train_step_dev): all instances take step
 * t = *step_counter + 1, then the counter is incremented on the stream. */
jet_status jet_batch_train_step_dev(jet_batch_t batch, void* const* params, void* const* adam_m,
                                    void* const* adam_v, int64_t* step_counter, float lr, const void* const* X,
                                    const int64_t* N, const void* const* source,
                                    double* loss_out /* device [n] or NULL */, jet_stream_t stream);
jet_status jet_batch_destroy(jet_batch_t batch);

/*
 * Verification hook for the transpose inner-product test of Eq. 15: applies
 * the plan's activation-jet rule elementwise in FP64 to n jets of C channels
 * (layout [n][C]):
 *   kind 0: out = compose(z)                 (a-jet of z, Eq. 2-3)
 *   kind 1: out = (d compose / dz)(z) v      (tangent)
 *   kind 2: out = (d compose / dz)(z)^T v    (adjoint used by the backward)
 * z, v, out: device double arrays.
 */
jet_status jet_debug_activation(jet_plan_t plan, int32_t kind, int64_t n, const double* z, const double* v,
                                double* out, jet_stream_t stream);

/*
 * Measurement hook.  While enabled, every call on the plan records a pair of
 * CUDA events on the call's stream around its dominant kernel (the fused jet
 * kernel).  jet_plan_profile_read synchronises on those events, returns the
 * number of recorded launches and their summed device time in milliseconds,
 * and clears the record.  Enabling costs two event records per call.
 */
jet_status jet_plan_profile(jet_plan_t plan, int32_t enable);
jet_status jet_plan_profile_read(jet_plan_t plan, int64_t* launches, double* total_ms);

/*
 * jet_backward_params without any device allocation (the paper has no
 * counterpart: this is a deployment convenience of this library).
 *
 * For callers that cannot call cudaMalloc -- runtimes that own every device
 * allocation themselves, or real-time loops that forbid allocator calls after
 * start-up -- and therefore cannot create a plan (jet_plan_create allocates
 * the plan's workspace).  It takes the jet_plan_create arguments (JET_FP64 or
 * JET_FP32 only) together with the jet_backward_params arguments, and keeps
 * all working memory (weight copies, per-chunk FP64 gradient slices,
 * per-CTA jet scratch) in one file-scope device array of 8 MiB that every
 * GPU loading the library reserves until the process exits.
 *   params, X, source, grad_out, loss_out: as jet_backward_params (device;
 *             the caller allocates them); N >= 1.
 *   scratch_bytes_used: optional host out-param, bytes of the array used.
 * Shapes whose working set exceeds 8 MiB even with a single chunk of tiles
 * are rejected with JET_ERR_UNSUPPORTED before any launch.
 * Set-up: the first call on each device looks up the array's device address
 * with cudaGetSymbolAddress (that device current) and caches it for the
 * later calls on that device.  Every call reuses the same array and leaves its
 * contents behind; each call writes every part it reads, so nothing has to be
 * cleared, but calls that overlap on the GPU (two streams or two host
 * threads) race on the array and must be serialised by the caller.
 */
jet_status jet_backward_params_noalloc(const jet_residual_spec* spec, int32_t d_in, int32_t n_layers,
                                       const int32_t* widths, int32_t n_needed, const jet_chan* needed,
                                       jet_precision prec, const void* params, const void* X, int64_t N,
                                       const void* source, void* grad_out, double* loss_out,
                                       jet_stream_t stream, size_t* scratch_bytes_used);

/*
 * Verification hook for failure detection: launches one CTA that waits on an
 * mbarrier nothing arrives at, with the same bounded wait the tensor-core
 * kernels use and a budget of budget_ns nanoseconds (1e3..1e9).  The kernel
 * gives up, records the time-out and returns; the call synchronises and
 * returns JET_ERR_TIMEOUT (the device context stays usable).  Any other
 * status means the bounded wait or its reporting is broken.
 */
jet_status jet_debug_wait_timeout(int64_t budget_ns);

/* Thread-local message for the last failing call on this thread. */
const char* jet_last_error(void);

/* Library version string. */
const char* jet_version(void);

#ifdef __cplusplus
}
#endif

#endif /* JET_H_ */
