// Internal layout shared by the host setup and the CUDA kernels of the solver.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace dlmpc {

constexpr int kMaxNx = 4;
constexpr int kMaxNu = 4;

// One column patch (Sec. III-D): the columns of global subsystem `sub`,
// together with every Phi row of the subsystems in Patch(sub).
struct Item {
  int32_t inst;       // instance index
  int32_t sub;        // global subsystem index
  int32_t n_mem;      // |Patch(sub)|
  int32_t mem_off;    // offset into members[] / rev_slot[]
  int32_t self_pos;   // position of `sub` inside its own patch
  int32_t r_sub;      // rows per subsystem
  int32_t T;
  int32_t dred;       // reduced variables: (r_sub - nx) * n_mem (slot-0 states removed)
  int32_t dred_pad;   // dred rounded up to a multiple of 4
  int32_t k;          // nullity of the restricted constraint
  int32_t kpad;       // odd row stride of N (>= k)
  int32_t mrows;      // kept constraint rows (reduced)
  int64_t n_off;      // float offset of N (dred_pad x kpad) and N^T (k x dred_pad), row-major
  int64_t q_off;      // float offset of q: nx x dred_pad
  int64_t st_off;     // float offset of the column-owned state: nx x (r_sub * n_mem)
  int64_t z_off;      // offset into the reduced constraint CSR row pointer array
  int64_t ws_off;     // double offset of the factorisation workspace
  // placement inside the sweep kernel's shared-memory arena of its CTA
  int32_t n_sm;       // resident N (float offset), or -1: streamed through the group buffer
  int32_t q_sm;       // resident q (float offset), or -1: read from global memory
  int32_t st_sm;      // resident Psi then Lambda (2 * nx * D_col floats), or -1: global memory
  int32_t lslot;      // slot of the item's instance among the instances of its CTA
  int64_t cp_off;     // float offset of the compact iterate (see cp_floats), global copy
  int32_t cp_sm;      // resident compact iterate (float offset), or -1: global memory
  int32_t cp_pad;
};

// Floats of the projection operator of one item: N (dred_pad x kpad) then
// N^T (k x dred_pad), both row-major.
inline __host__ __device__ unsigned n_floats(const Item &it) {
  return (unsigned)(it.dred_pad * it.kpad + it.k * it.dred_pad);
}

// Compact iterate of one item (iterations after the first of a launch):
// lhat [round4(D_col)] (reduced rows, then slot-0 rows), R [dred_pad],
// Y [kpad], t0 [nx][kpad].
inline __host__ __device__ int cp_floats(const Item &it, int nx) {
  return ((it.r_sub * it.n_mem + 3) & ~3) + it.dred_pad + (1 + nx) * it.kpad;
}

// Arguments of the persistent ADMM sweep kernel.
struct Params {
  const Item *items;
  int32_t n_items;
  const int32_t *grp_ptr;     // [grid * ng + 1]: items of group g of CTA b are
  const int32_t *grp_items;   //   grp_items[grp_ptr[b * ng + g] .. grp_ptr[b * ng + g + 1])
  const int32_t *cta_inst_ptr;// [grid + 1]: instances touched by CTA b (local slot order)
  const int32_t *cta_inst;
  const int32_t *members;     // global subsystem ids of every patch, per item at mem_off
  const int32_t *rev_slot;    // slot of the item's subsystem within Patch(member)
  const int32_t *np_of;       // |Patch(i)| per global subsystem
  const int64_t *g_off;       // exchange-buffer offset of row-subsystem i (np_of[i] x r_sub floats)
  const float *Nmat;
  const float *qvec;
  float *Psi;
  float *Lam;
  float *Phi;                 // optional export (may be null)
  float *G0;
  float *G1;
  float *S;                   // ||x_hat_i||^2 per global subsystem
  const float *x;
  float *u;
  float *x_next;
  // per global subsystem parameters
  const float *qw;            // [sub][nx]
  const float *rw;            // [sub][nu]
  const float *xlo, *xhi;     // [sub][nx]
  const float *ulo, *uhi;     // [sub][nu]
  const double *Adiag;        // [sub][nx][nx]
  const double *Aoff;         // [nnz][nx][nx]
  const int32_t *adj_ptr;     // global CSR (indices global)
  const int32_t *adj_idx;
  const double *Bm;           // [sub][nx][nu]
  int32_t n_inst;
  const float *rho_i, *epsp_i, *epsd_i;  // per instance
  unsigned long long *bar;    // [3] barrier counters: arrivals (low 32 bits) + not-converged items (high 32)
  unsigned int *notconv;      // [3][n_inst] not-converged items per instance (used when n_inst > 1)
  int32_t *inst_iters;        // [n_inst]
  int32_t *conv_prev;         // [n_inst] != 0: the instance's last step met Conv (DLMPC_WARM_CONVERGED)
  float *item_r, *item_s;     // [n_items]
  int32_t *err;               // [8]: code, cta, iteration, aux, iterations run
  int32_t max_iter;
  int32_t fixed_iters;
  int32_t warm;               // 0 cold, 1 previous
  int32_t nx, nu;
  unsigned long long timeout_ns;
  // launch shape and shared-memory arena (floats)
  int32_t ng;                 // thread groups per CTA
  int32_t wave;               // items whose Phi-step is batched per group
  int32_t max_dcol, max_dred_pad, max_kpad, max_nmem;
  int32_t grp_floats;         // floats per group region
  int32_t cta_floats;         // floats of the per-CTA counters (after the group regions)
  int32_t max_local_inst;
  int32_t rows_cached;        // != 0: every group holds one wave; row records kept in shared memory
  unsigned long long *trace;  // optional [grid][kTraceIters][kTracePoints] globaltimer stamps
  int32_t skip_arrival_cta;   // test of the bounded waits: this CTA leaves before its first
                              // iteration barrier (-1 = none)
  int32_t compact;            // != 0: iterations after the first use the compact iterate
  // simulated lost messages: the row sums patch j sends to member m at the end
  // of iteration k are lost when SplitMix64 draw (k N + j) N + m of stale_seed,
  // shifted right by 11, is below stale_thr (0: none); the receiver keeps the
  // value it holds
  unsigned long long stale_thr, stale_seed;
  int32_t block_cost;         // != 0: Phi-step by slot box-QP with the full cost blocks
  const float *qblk2, *rblk2; // [sub][nx][nx] 2 Q_i, [sub][nu][nu] 2 R_i
  // explicit solution of the slot QP with coupled rows (null: boxes only);
  // key = 2 * global subsystem + kind (0 state slots, 1 input slots)
  float *expl;                // [regions][expl_stride]: K [n][n], k [n], L [n][n], l [n] (z = K w + k, mu = L w + l)
  const int32_t *rg_base, *rg_cnt;  // per key: first region, region count
  const int32_t *rw_base, *rw_cnt;  // per key: first constraint row, row count
  const uint32_t *rg_desc;    // per region: active-row count (bits 0..3), row indices (4 bits each)
  const float *crow;          // [rows][crow_stride]: unit normal [nmax], right-hand side
  int32_t expl_stride, crow_stride;
  float *cpst;                // compact iterates of the items without shared-memory residency
};

constexpr int kTraceIters = 8;
constexpr int kTracePoints = 8;

// Reduced constraint system of one item for the one-time factorisation:
// CSR over the kept rows of Z_j restricted to the non-slot-0 variables, and
// the right-hand sides b_c (per own column c) over the same rows.
struct FactorParams {
  const Item *items;
  int32_t n_items;
  const int64_t *zrow_ptr;    // per item: mrows+1 entries starting at z_off (absolute nnz offsets)
  const int32_t *zcol;
  const double *zval;
  const double *rhs;          // per item: nx x mrows, starting at rhs_off[item]
  const int64_t *rhs_off;
  double *ws;                 // per-concurrent-CTA workspace
  int64_t ws_stride;          // doubles per CTA workspace
  float *Nmat;
  float *qvec;
  double *feas;               // [n_items] max_c ||Z q_c - b_c||_inf
  int32_t *rank;              // [n_items]
  int32_t *nullity;           // [n_items] k actually found (must equal planned k)
  int32_t nx;
  const int32_t *order;       // [n_items] patches by decreasing work (the queue)
  int32_t *next;              // queue position (zero before the launch)
  int32_t use_smem;           // workspace in dynamic shared memory
};

}  // namespace dlmpc
