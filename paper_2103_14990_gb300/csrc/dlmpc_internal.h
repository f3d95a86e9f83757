// Internal layout shared by the host setup and the CUDA kernels of the solver.
#pragma once
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
  int64_t n_off;      // float offset of N: dred_pad x kpad, row-major
  int64_t q_off;      // float offset of q: nx x dred_pad
  int64_t st_off;     // float offset of the column-owned state: nx x (r_sub * n_mem)
  int64_t z_off;      // offset into the reduced constraint CSR row pointer array
  int64_t ws_off;     // double offset of the factorisation workspace
};

struct Params {
  const Item *items;
  int32_t n_items;
  const int32_t *cta_ptr;     // [grid+1] items of CTA b: cta_items[cta_ptr[b] .. cta_ptr[b+1])
  const int32_t *cta_items;
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
  unsigned int *bar;          // grid barrier counter
  unsigned int *notconv;      // [3][n_inst+1]
  int32_t *inst_iters;        // [n_inst]
  float *item_r, *item_s;     // [n_items]
  int32_t *err;               // [8]: code, cta, iteration, aux, iterations run
  int32_t max_iter;
  int32_t fixed_iters;
  int32_t warm;               // 0 cold, 1 previous
  int32_t nx, nu;
  unsigned long long timeout_ns;
  int32_t smem_n_floats;      // floats of shared memory reserved for N chunks
};

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
  int32_t item_begin;         // items item_begin .. item_begin+gridDim.x-1 in this launch
  int32_t use_smem;           // workspace in dynamic shared memory
};

}  // namespace dlmpc
