/*
 * dlmpc.h - C ABI of the GB300 DLMPC solver.
 *
 * Distributed and localized MPC (Sec. II-A): at every MPC step (Alg. 1) an ADMM
 * over the system-level parameterisation Phi runs until convergence (Alg. 2):
 *   Phi-comp     row-wise box-QP on Phi x(tau)          (Alg. 2, Phi-comp)
 *   Psi-comp     column-wise projection onto Z_AB Psi = I within the d-hop patch
 *   Lambda-comp  Lambda <- Lambda + Phi - Psi
 *   Conv         per-subsystem primal/dual residuals, global AND
 * and the first input slot of Phi x(tau) is applied: x(tau+1) = A x + B u.
 *
 * Conventions shared by every entry point:
 *  - One context holds n_inst >= 1 independent instances; all share nx and nu,
 *    T and d may differ.  Subsystems of all instances are concatenated in
 *    instance order ("global subsystem index").
 *  - Phi has T state slots (t = 0..T-1) and T-1 input slots per subsystem:
 *    r_sub = nx*T + nu*(T-1) rows per subsystem (Sec. II-A, shape of Phi).
 *  - Locality: Phi(row of i, column of j) may be nonzero iff the hop distance
 *    of i and j on the coupling graph is <= d.  Patch(j) lists those i in
 *    ascending order.
 *  - Column-owned state layout (get/set_state): for every global subsystem j,
 *    for every own column c < nx, for every member m of Patch(j) (ascending),
 *    for every local row r < r_sub: one float.  Local rows are ordered state
 *    slot-major (t*nx + a for t < T), then inputs (nx*T + t*nu + b).
 *  - Pointers named *_dev are device pointers that must be valid on the
 *    context's stream; every other pointer is host memory.  The caller keeps
 *    ownership of everything it passes; the library copies setup inputs and
 *    owns all its workspaces.
 *  - Return codes: 0 = OK, > 0 soft status, < 0 error.  No C++ exception or
 *    abort crosses this boundary; dlmpc_last_error() explains the last error.
 *  - Calls are asynchronous on the context's stream unless they return host
 *    statistics, which synchronise on that stream.
 */
#ifndef DLMPC_H
#define DLMPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DLMPC_OK 0
#define DLMPC_MAX_ITER 1                 /* ADMM stopped at max_iter; results still written */
#define DLMPC_ERR_ARG (-1)               /* invalid argument or call order */
#define DLMPC_ERR_INFEASIBLE_LOCALITY (-2) /* some Z_j psi = e_c has no solution */
#define DLMPC_ERR_NONFINITE (-3)         /* NaN/Inf residual during ADMM */
#define DLMPC_ERR_TIMEOUT (-4)           /* a device-side wait gave up (bounded spin) */
#define DLMPC_ERR_CUDA (-5)              /* a CUDA runtime call failed */
#define DLMPC_ERR_NOMEM (-6)             /* device allocation failed */
#define DLMPC_ERR_CAPACITY (-7)          /* an output buffer is smaller than the result; the
                                            sizes needed are reported beside it */

#define DLMPC_WARM_COLD 0      /* Psi = Lambda = 0 */
#define DLMPC_WARM_PREVIOUS 1  /* continue from the state left by the previous step/set_state */
#define DLMPC_WARM_LEARNED 2   /* learned initial Phi rows and Lambda, then a Psi-step first */
#define DLMPC_WARM_CONVERGED 3 /* per instance: the previous step's state if that step met Conv
                                  (or the state came from dlmpc_set_state), zeros otherwise: a step
                                  stopped at max_iter is a worse start than zeros */

typedef struct dlmpc_ctx dlmpc_ctx;
typedef struct dlmpc_mlp dlmpc_mlp;

/* One DLMPC instance: Eq. (MPC) of Sec. II-A with Q_t = Q, R_t = R for all t.
 * The coupling graph G_(A,B) is undirected, CSR, without self loops; column
 * indices ascending within each row.  Bounds apply to states of slots 1..T-1
 * and to all inputs; NULL means unbounded. */
typedef struct {
  int32_t n_sub, nx, nu, T, d;
  const int32_t *adj_ptr;   /* [n_sub+1] */
  const int32_t *adj_idx;   /* [adj_ptr[n_sub]] */
  const double *A_diag;     /* [n_sub][nx][nx] row-major A_ii */
  const double *A_off;      /* [nnz][nx][nx]   A_{i,adj_idx[e]} for CSR entry e of row i */
  const double *B;          /* [n_sub][nx][nu] B_ii (B block diagonal) */
  const double *q;          /* [n_sub][nx] diagonal of Q_i (> 0) */
  const double *r;          /* [n_sub][nu] diagonal of R_i (> 0) */
  const double *x_lo, *x_hi;/* [n_sub][nx] or NULL */
  const double *u_lo, *u_hi;/* [n_sub][nu] or NULL; 0 must lie in [u_lo, u_hi] */
  double rho;               /* ADMM penalty (> 0) */
  double eps_p, eps_d;      /* Conv thresholds on the per-subsystem residuals */
  int32_t max_iter;         /* ADMM iteration cap (>= 1) */
  /* Full cost blocks (Sec. II-A with non-diagonal Q_t = Q, R_t = R), or NULL:
   * [n_sub][nx][nx] Q_i and [n_sub][nu][nu] R_i, row-major, symmetric positive
   * definite; when given they replace q / r.  The Phi-step then solves, per
   * subsystem and time slot, the box-QP of the slot's nx (or nu) rows exactly. */
  const double *Q_blk;
  const double *R_blk;
  /* Coupled constraints of one subsystem at one time slot, beside the boxes
   * (Sec. II-A: the Phi-comp then has a piecewise-affine explicit solution,
   * precomputed at every MPC step from x(tau) as in Alg. 1):
   *   Gx[i] x_t <= gx[i]  on the state slots t = 1..T-1,
   *   Gu[i] u_t <= gu[i]  on every input slot,
   * Gx [n_sub][n_cx][nx], gx [n_sub][n_cx], Gu [n_sub][n_cu][nu],
   * gu [n_sub][n_cu], row-major; n_cx, n_cu in 0..DLMPC_MAX_COUPLED (the
   * pointers may be NULL when the count is 0).  Every row needs a nonzero
   * normal and g >= 0, so that 0 satisfies the slot's rows and the box.
   * Rows are normalised to unit normals on upload.  With coupled rows the
   * Phi-step is the slot QP (as with Q_blk / R_blk); a slot with more than
   * DLMPC_MAX_REGIONS candidate active sets is rejected. */
  int32_t n_cx, n_cu;
  const double *Gx, *gx;
  const double *Gu, *gu;
} dlmpc_problem;

#define DLMPC_MAX_COUPLED 4     /* coupled rows per subsystem and slot kind */
#define DLMPC_MAX_REGIONS 1024  /* active sets (explicit-solution regions) per subsystem and slot kind */

/* Per-instance result of one MPC step. */
typedef struct {
  int32_t iters;            /* ADMM iterations run */
  int32_t status;           /* DLMPC_OK (converged) or DLMPC_MAX_ITER */
  float r_max;              /* max_j ||Phi - Psi||_F over j's columns, last iteration */
  float s_max;              /* max_j rho ||Psi^{k+1} - Psi^k||_F over j's columns */
} dlmpc_stats;

/* Sizes of a context (host struct filled by dlmpc_get_info). */
typedef struct {
  int32_t n_inst, n_sub_total, nx, nu;
  int32_t n_items;          /* column patches = n_sub_total */
  int32_t max_dcol, max_nullity;
  int64_t state_floats;     /* floats of one column-owned matrix (Phi, Psi or Lambda) */
  int64_t operator_bytes;   /* bytes of all null-space bases N_j and their transposes (FP32, padded) */
  int64_t offset_bytes;     /* bytes of all min-norm offsets q_c (FP32, padded) */
  int64_t exchange_floats;  /* floats of one row-partial-sum exchange buffer */
  int32_t grid_ctas, threads_per_cta, smem_bytes; /* launch of the ADMM sweep kernel */
  int32_t group_threads, groups_per_cta, wave; /* sweep shape (DLMPC_OPT_SWEEP_SHAPE) */
  int32_t resident_n_items;     /* patches whose N_j stays in shared memory for the whole step */
  int32_t resident_state_items; /* patches whose Psi, Lambda and q stay in shared memory */
  int64_t iter_bytes;       /* bytes the sweep kernel's own loads move in one compact ADMM
                               iteration over all patches: N_j and its stored transpose
                               N_j^T read once each, row partial sums read (|Patch(m)| per
                               patch row) and written, the compact iterate (lhat, R, Y)
                               read and written */
  int64_t iter_bytes_min;   /* algorithmic bytes of the same iteration (the roofline's
                               numerator): as iter_bytes with every N_j counted once (both
                               products N_j^T alpha and N_j y read the same entries) */
} dlmpc_info;

/* Option keys for dlmpc_set_option. */
#define DLMPC_OPT_FIXED_ITERS 1   /* > 0: run exactly this many iterations, Conv only reported */
#define DLMPC_OPT_MAX_ITER 2      /* overrides every instance's max_iter */
#define DLMPC_OPT_TIMEOUT_MS 3    /* bound of every device-side wait (default 2000) */
#define DLMPC_OPT_EXPORT_PHI 4    /* != 0: keep the last Phi for dlmpc_get_state */
#define DLMPC_OPT_SWEEP_SHAPE 5   /* sweep launch: threads per group (64, 96, 128 or 256) * 10000
                                     + groups per CTA (1..15, at most 1024 threads) * 100
                                     + Phi-step wave (e.g. 1280402); replans the launch */
#define DLMPC_OPT_TIMING 7        /* != 0: record CUDA events around every step (dlmpc_get_timing) */
#define DLMPC_OPT_TRACE 9         /* != 0: record phase timestamps of the sweep (dlmpc_get_trace) */
#define DLMPC_OPT_GRAPH 10        /* != 0: run each step as a CUDA graph (captured on first use for
                                     a given set of buffers and options, then replayed); with it,
                                     dlmpc_get_timing reports the whole step in both fields */
#define DLMPC_OPT_LEARN_PLANT 11  /* != 0: network inputs also carry each patch member's A_mm and
                                     summed coupling blocks (set before dlmpc_attach_mlp) */
#define DLMPC_OPT_TEST_SKIP_ARRIVAL 12 /* test of failure handling: CTA `value` of the sweep leaves
                                          before its first iteration barrier, so every other CTA's
                                          bounded wait runs out and the step returns
                                          DLMPC_ERR_TIMEOUT (-1 = off, the default) */
#define DLMPC_OPT_RESIDENCY 8     /* shared-memory residency during a step: 0 none (all streamed),
                                     1 compact iterate, Psi/Lambda and q, 2 (default) also N where
                                     it fits; replans */
#define DLMPC_OPT_BLOCK_PHI 14    /* != 0: use the slot box-QP Phi-step even when every cost
                                     block is diagonal (it is used whenever one is not) */
#define DLMPC_OPT_STALE_PROB 15   /* probability p in [0, 1] that a message is lost (default 0),
                                     simulating the fully distributed setting (Sec. V): the row
                                     sums patch j sends to member m at the end of iteration k are
                                     lost when output n = (k N + j) N + m of SplitMix64 seeded with
                                     DLMPC_OPT_STALE_SEED, shifted right by 11 bits, is below
                                     floor(p 2^53) (N = subsystems of the context, j, m global
                                     indices); the receiver keeps the last value it received (the
                                     start state's before the first iteration) */
#define DLMPC_OPT_STALE_SEED 16   /* seed of those draws (a non-negative integer, default 0) */
#define DLMPC_OPT_COMPACT 13      /* != 0 (default): iterations after the first of a step carry the
                                     projected iterate as Psi = q + N t and Lambda = x_c lhat (the
                                     same iterates as Alg. 2, with the v = Psi + alpha x algebra of
                                     Psi-comp done once per patch instead of once per column);
                                     0: every iteration projects the stored Psi/Lambda.  Ignored
                                     (full form) while DLMPC_OPT_EXPORT_PHI is on. */

/* Builds the locality structure (hop-distance BFS, Patch(j), rows of Z_AB that
 * touch each patch) for n_inst instances, copies all inputs to the device and
 * allocates workspaces.  Sec. III-B "Setup".  probs: host array [n_inst].
 * stream: a cudaStream_t (NULL = legacy default stream).  On success *out
 * receives a context to be released with dlmpc_destroy. */
int dlmpc_setup(const dlmpc_problem *probs, int32_t n_inst, void *stream, dlmpc_ctx **out);

/* One-time precomputation (Alg. 1, first line; Sec. IV-C "Precomputation"):
 * for every column patch j, an FP64 pivoted Householder QR of the restricted
 * constraint matrix gives an orthonormal null-space basis N_j and the min-norm
 * offsets q_c = Z_j^+ e_c (stored FP32).  Returns DLMPC_ERR_INFEASIBLE_LOCALITY
 * if max_c ||Z_j q_c - e_c|| exceeds 1e-9 for some j. Synchronous. */
int dlmpc_precompute(dlmpc_ctx *ctx);

/* Plant update in place (Sec. IV-C: the precomputation dominates the GPU time
 * at large N, and Sec. V: a model that changes while the network runs).
 * n_changed subsystems (global indices over the context's instances, each at
 * most once) get new rows of the dynamics: A_diag (n_changed x nx x nx, the
 * new A_ii in the order of `subsystems`), A_off (for each changed subsystem
 * in that order, the nx x nx blocks A_ij of its adjacency entries in CSR
 * order; may be NULL when none has neighbours) and B (n_changed x nx x nu).
 * The coupling graph, costs and bounds stay.  Only the column patches whose
 * constraint rows see a changed subsystem (hop distance <= d + 1) are
 * re-factorised, in FP64 as dlmpc_precompute, and their N_j, N_j^T and q_c
 * replaced in place; all other operators, the iterates, options, launch plan
 * and captured graphs stay valid, and the next steps use the new dynamics.
 * All pointers are host pointers, copied.  Returns the number of patches
 * re-factorised (>= 0); DLMPC_ERR_INFEASIBLE_LOCALITY when a patch's
 * restricted constraint has no solution, DLMPC_ERR_ARG when a patch's
 * null-space dimension changes (the operator layout is fixed at precompute:
 * set up a new context for that plant) or for invalid arguments; on any
 * error the context is left as it was.  Synchronous. */
int dlmpc_update_plant(dlmpc_ctx *ctx, int32_t n_changed, const int32_t *subsystems, const double *A_diag,
                       const double *A_off, const double *B);

/* Checkpoint of the one-time precomputation (the paper has no counterpart):
 * dlmpc_export_operators writes every patch's null-space dimension, N_j, N_j^T
 * and q_c into the host buffer buf (cap bytes) and returns the blob's size;
 * with buf NULL or cap too small it only returns the size.
 * dlmpc_import_operators replaces dlmpc_precompute on a context set up with
 * the same problem structure (sizes, graphs, T, d; checked by a signature),
 * from a host blob of `size` bytes; DLMPC_ERR_ARG for a blob of another
 * structure or a truncated one.  Both synchronous; the caller owns buf. */
int64_t dlmpc_export_operators(dlmpc_ctx *ctx, void *buf, int64_t cap);
int dlmpc_import_operators(dlmpc_ctx *ctx, const void *buf, int64_t size);

/* One MPC step for every instance (Alg. 1 body): per-step precompute from
 * x(tau), ADMM to convergence (Alg. 2), u(tau) = slot-0 inputs of Phi x(tau),
 * x(tau+1) = A x(tau) + B u(tau).
 * x_dev: [n_sub_total][nx] float; u_dev: [n_sub_total][nu] float (written);
 * x_next_dev: [n_sub_total][nx] float or NULL.  warm: DLMPC_WARM_*.
 * stats: host [n_inst] or NULL (NULL keeps the call asynchronous).
 * Returns the worst status over instances (DLMPC_MAX_ITER if any hit the cap)
 * or an error. */
int dlmpc_step(dlmpc_ctx *ctx, const float *x_dev, float *u_dev, float *x_next_dev,
               int32_t warm, dlmpc_stats *stats);

/* Same as dlmpc_step with one device buffer per instance: x_dev[b], u_dev[b],
 * x_next_dev[b] (host arrays of n_inst device pointers; x_next_dev may be NULL). */
int dlmpc_solve_batch(dlmpc_ctx *ctx, const float *const *x_dev, float *const *u_dev,
                      float *const *x_next_dev, int32_t warm, dlmpc_stats *stats);

/* Same as dlmpc_step with HOST buffers: copies x to the device, runs the step,
 * copies u (and x_next if non-NULL) back, then synchronises. */
int dlmpc_step_host(dlmpc_ctx *ctx, const float *x, float *u, float *x_next,
                    int32_t warm, dlmpc_stats *stats);

int dlmpc_set_option(dlmpc_ctx *ctx, int32_t key, double value);
int dlmpc_get_info(dlmpc_ctx *ctx, dlmpc_info *info);

/* Copies the state (device pointers, column-owned layout, info.state_floats
 * floats each; any may be NULL).  phi needs DLMPC_OPT_EXPORT_PHI. */
int dlmpc_get_state(dlmpc_ctx *ctx, float *phi_dev, float *psi_dev, float *lam_dev);
/* Replaces Psi and Lambda (device pointers, same layout); used by
 * DLMPC_WARM_PREVIOUS and DLMPC_WARM_CONVERGED on the next step. */
int dlmpc_set_state(dlmpc_ctx *ctx, const float *psi_dev, const float *lam_dev);

/* Host copy of Patch(j) of global subsystem j (members as global indices);
 * returns |Patch(j)| or an error.  cap = capacity of members. */
int dlmpc_get_patch(dlmpc_ctx *ctx, int32_t j, int32_t *members, int32_t cap);

/* Host copy of the precomputed operator of column patch j in the FULL
 * column-owned variable order (D_col = r_sub*|Patch(j)| rows): N (D_col x k,
 * row-major, slot-0 state rows zero) and q (nx x D_col).  Returns k. */
int dlmpc_get_operator(dlmpc_ctx *ctx, int32_t j, double *N, int32_t n_cap,
                       double *q, int32_t q_cap);

/* Sweep phase timestamps of the last step (needs DLMPC_OPT_TRACE): for every
 * CTA, the first 8 iterations, 8 %globaltimer stamps (ns) taken by thread 0:
 * 0 iteration start, 1 first Phi-step wave done, 2 first patch projected,
 * 3 last patch done, 4 all groups done, 5 grid barrier passed (0 = not taken).
 * stamps: host [cap]; returns the number of CTAs.  Synchronous. */
int dlmpc_get_trace(dlmpc_ctx *ctx, unsigned long long *stamps, int64_t cap);

/* GPU time of the last step, from CUDA events recorded on the context's
 * stream (needs DLMPC_OPT_TIMING): ms[0] = the ADMM sweep kernel alone,
 * ms[1] = the whole step (first memset to the end of the statistics copy).
 * Waits for the step to finish. */
int dlmpc_get_timing(dlmpc_ctx *ctx, float *ms);

/* Allocation-free re-factorisation of one patch constraint block.  The paper
 * has no counterpart: it serves callers that must not allocate device memory
 * once their control loop runs, such as a real-time MPC thread refreshing the
 * patches touched by a model update between two steps (cudaMalloc may
 * synchronise the whole device and its latency is unbounded), or code that is
 * limited to a memory budget fixed at start-up.
 * Computes in FP64 what dlmpc_precompute computes for one column patch: from
 * the constraint block Z_dev (m x D, row-major) and nrhs right-hand sides
 * rhs_dev (nrhs x m), an orthonormal null-space basis N_dev (D x k_cap,
 * row-major; the first `nullity` columns are written, the others zeroed), the
 * min-norm solutions q_dev (nrhs x D), rank_nullity_dev[2] = {rank, nullity}
 * and feas_dev[0] = max_c ||Z q_c - rhs_c||_inf.  All pointers are device
 * pointers owned by the caller; nothing is allocated.
 * Workspace: one static device array of DLMPC_NOALLOC_MAX_DOUBLES doubles
 * (8 MiB), held by every GPU that loads the library until the process exits.
 * A block needing more than that (D*m + (3+nrhs)*m + 8*D + (m+1)/2 doubles,
 * integer division) or nrhs > 32 returns DLMPC_ERR_ARG without launching
 * anything.  The array's device address is looked up on the first call on
 * each device, with that device current; make that first call before any
 * stream capture.  Every call uses the same array: calls that overlap on the
 * GPU race, so serialise them.
 * Runs on `stream` (a cudaStream_t, NULL = legacy default stream) and waits
 * for it: the call reads {rank, nullity} back (8 bytes into host stack
 * memory) and returns DLMPC_ERR_CAPACITY when nullity > k_cap, in which case
 * N_dev holds the first k_cap basis columns and rank_nullity_dev the true
 * sizes; DLMPC_ERR_CUDA if the launch or the wait fails. */
#define DLMPC_NOALLOC_MAX_DOUBLES (1 << 20)
int dlmpc_factor_patch_noalloc(const double *Z_dev, int32_t m, int32_t D, const double *rhs_dev,
                               int32_t nrhs, double *N_dev, int32_t k_cap, double *q_dev,
                               int32_t *rank_nullity_dev, double *feas_dev, void *stream);

/* ---- learned warm start (Sec. V names a better ADMM starting point as future
 * work; the network and its training are this library's, not the paper's) ----
 *
 * Network: x -> GELU(x W1 + b1) -> GELU(. W2 + b2) -> . W3 + b3, BF16 tensor-core
 * GEMMs with FP32 accumulation, FP32 master parameters, AdamW.  Parameter
 * block (FP32, in this order): W1 [d_in][hidden], b1 [hidden], W2
 * [hidden][hidden], b2 [hidden], W3 [hidden][d_out], b3 [d_out]; row-major.
 * The network predicts normalised outputs; forward returns y * scale + shift.
 * Create the network on the same stream as the contexts it serves. */
int dlmpc_mlp_create(int32_t d_in, int32_t hidden, int32_t d_out, void *stream, dlmpc_mlp **out);
int64_t dlmpc_mlp_num_params(dlmpc_mlp *mlp);
/* Sets the parameters (host, num_params floats) and the output scale/shift
 * (host [d_out] each, NULL keeps them); resets the AdamW moments. */
int dlmpc_mlp_set_params(dlmpc_mlp *mlp, const float *params, int64_t n, const float *out_scale,
                         const float *out_shift);
int dlmpc_mlp_get_params(dlmpc_mlp *mlp, float *params, int64_t n);
/* y_dev [n][d_out] = de-normalised network output for x_dev [n][d_in] (device). */
int dlmpc_mlp_forward(dlmpc_mlp *mlp, const float *x_dev, int32_t n, float *y_dev);
/* Mean squared error against normalised targets t_dev [n][d_out] and its
 * gradient w.r.t. every parameter (grad_host [num_params], may be NULL). */
int dlmpc_mlp_gradients(dlmpc_mlp *mlp, const float *x_dev, const float *t_dev, int32_t n, float *grad_host,
                        double *loss_host);
/* One AdamW step (beta1 0.9, beta2 0.999, eps 1e-8, decoupled weight decay)
 * on the batch; loss_host (may be NULL) receives the batch loss before it. */
int dlmpc_mlp_train_step(dlmpc_mlp *mlp, const float *x_dev, const float *t_dev, int32_t n, float lr,
                         float weight_decay, double *loss_host);
const char *dlmpc_mlp_last_error(dlmpc_mlp *mlp);
void dlmpc_mlp_destroy(dlmpc_mlp *mlp);

/* Widths of the network input (patch state of a subsystem, members placed by
 * position relative to it, zero padded) and output (its Phi rows then its
 * Lambda rows over the same member slots: 2 * r_sub * slots * nx). */
int dlmpc_learned_dims(dlmpc_ctx *ctx, int32_t *d_in, int32_t *d_out);
/* feats_dev [n_sub_total][d_in] from x_dev (device). */
int dlmpc_learned_features(dlmpc_ctx *ctx, const float *x_dev, float *feats_dev);
/* targets_dev [n_sub_total][d_out]: the rows of the last Phi (needs
 * DLMPC_OPT_EXPORT_PHI during the step) and of Lambda. */
int dlmpc_learned_targets(dlmpc_ctx *ctx, float *targets_dev);
/* Network used by DLMPC_WARM_LEARNED (NULL detaches): each step then starts
 * from Psi0 = proj(Phi~ + Lambda~), Lambda0 = Lambda~ + Phi~ - Psi0. */
int dlmpc_attach_mlp(dlmpc_ctx *ctx, dlmpc_mlp *mlp);

/* Ablation of the paper's GPU mappings (Sec. III): variant 0 = naive (one
 * kernel per ADMM step, thread per row/column/element, every step's result
 * shared through host memory, Conv flag read each iteration, Sec. III-A);
 * 1 = combined (Phi kernel, then one Psi+Lambda+Conv kernel per column, one
 * host exchange per iteration, Sec. III-C); 2 = the persistent column-patch
 * sweep of this library.  Runs exactly `iters` iterations from `warm`
 * (COLD or PREVIOUS) on x_dev, leaves Phi (allocating it if needed), Psi and
 * Lambda in the context, and writes the host wall time to *ms_out.
 * Requires null-space dimensions <= 256.  Synchronous. */
int dlmpc_run_variant(dlmpc_ctx *ctx, int32_t variant, const float *x_dev, int32_t iters, int32_t warm,
                      double *ms_out);

/* One measured launch shape of the sweep kernel. */
typedef struct {
  int32_t group_threads, groups_per_cta, wave, residency;
  float ms;                 /* best sweep-kernel time of `iters` iterations */
} dlmpc_tune_entry;

/* Autotuner of the sweep launch (A7): for every feasible combination of
 * threads per group, groups per CTA, Phi-step wave and shared-memory
 * residency, runs `iters` fixed ADMM iterations from a cold start on x_dev
 * (device, [n_sub_total][nx]), times the kernel with CUDA events, keeps the
 * fastest plan and caches it per problem signature for the process.
 * A plan's one-time prologue (bulk copies of resident N) is part of each
 * timing, so `iters` near the steps' own iteration count ranks the plans as
 * the steps will see them.
 * iters <= 0 applies the cached choice without measuring.  Psi and Lambda are
 * restored afterwards.  entries (host, may be NULL) receives up to `cap`
 * measured shapes.  Returns the number measured, or an error.  Synchronous. */
int dlmpc_autotune(dlmpc_ctx *ctx, const float *x_dev, int32_t iters, dlmpc_tune_entry *entries, int32_t cap);

const char *dlmpc_last_error(dlmpc_ctx *ctx);
void dlmpc_destroy(dlmpc_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* DLMPC_H */
