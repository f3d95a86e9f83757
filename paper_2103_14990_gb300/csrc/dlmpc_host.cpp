// Host side of the DLMPC solver: locality structure (Sec. II-A, d-hop
// patches), the reduced per-patch constraint systems, work assignment and the
// C ABI declared in include/dlmpc.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <tuple>
#include <limits>
#include <map>
#include <mutex>
#include <numeric>
#include <queue>
#include <string>
#include <vector>

#include "dlmpc_internal.h"
#include "../../include/dlmpc.h"

#include <nvtx3/nvToolsExt.h>

namespace dlmpc {
cudaError_t launch_factor(const FactorParams &p, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_repack(const Item *scratch_items, const Item *items, int n_items, const float *src, float *dst,
                          cudaStream_t s);
const void *sweep_kernel_ptr(int nx, int gt, bool blk, int threads);
int sweep_group_floats(int nx, int nu, int gt, int wave, int max_dcol, int max_dred_pad, int max_kpad, int max_nmem,
                       bool rows_cached);
cudaStream_t mlp_stream(const dlmpc_mlp *mlp);
cudaError_t launch_sweep(const Params &P, int gt, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_stats(const int32_t *inst_item_ptr, int n_inst, const float *item_r, const float *item_s,
                         const int32_t *inst_iters, const int32_t *err, int fixed, const float *epsp,
                         const float *epsd, dlmpc_stats *out, cudaStream_t s);
cudaError_t launch_gather(const float *const *src, const int32_t *off, int n_inst, int width, float *dst,
                          cudaStream_t s);
struct LearnArgs {
  const Item *items;
  int n_items;
  const int32_t *members;
  const int32_t *rev_slot;
  int nx, slots, L, max_rsub;
  int d_out;
  int plant;
  const double *Adiag, *Aoff;
  const int32_t *adj_ptr;
};
cudaError_t launch_learn_features(const LearnArgs &A, const float *x, float *feats, cudaStream_t s);
struct VariantArgs {
  const Item *items;
  int n_items;
  const int32_t *members;
  const int32_t *rev_slot;
  const float *Nmat, *qvec;
  float *Phi, *Psi, *Lam, *PsiPrev;
  const float *x;
  float *S;
  const float *qw, *rw, *xlo, *xhi, *ulo, *uhi;
  const float *rho_i, *epsp_i, *epsd_i;
  int nx, nu;
  unsigned *notconv;
};
cudaError_t launch_variant_s(const VariantArgs &A, cudaStream_t s);
cudaError_t launch_variant_phi(const VariantArgs &A, const int32_t *row_sub, const int32_t *row_loc, int total,
                               cudaStream_t s);
cudaError_t launch_variant_psi(const VariantArgs &A, cudaStream_t s);
cudaError_t launch_variant_lambda(const VariantArgs &A, int64_t n, cudaStream_t s);
cudaError_t launch_variant_conv(const VariantArgs &A, cudaStream_t s);
cudaError_t launch_variant_combined(const VariantArgs &A, cudaStream_t s);
cudaError_t launch_learn_rows(const LearnArgs &A, float *phi, float *lam, float *rows, int dir, cudaStream_t s);
cudaError_t launch_learn_init(const Item *items, int n_items, int nx, int max_dred, int max_kpad, const float *Nmat,
                              const float *qvec, const float *phi, float *psi, float *lam, cudaStream_t s);
cudaError_t launch_scatter(const float *src, const int32_t *off, int n_inst, int width, float *const *dst,
                           cudaStream_t s);
}  // namespace dlmpc

using namespace dlmpc;

namespace {

thread_local std::string g_setup_error;

template <class T>
struct DevBuf {
  T *p = nullptr;
  size_t n = 0;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  cudaError_t alloc(size_t count) {
    release();
    n = count;
    if (count == 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void **>(&p), count * sizeof(T));
  }
};

struct Instance {
  int n_sub = 0, T = 0, d = 0, sub_off = 0, item_off = 0;
  std::vector<int32_t> adj_ptr, adj_idx;
  std::vector<double> A_diag, A_off, B, q, r, x_lo, x_hi, u_lo, u_hi;
  std::vector<double> Qb, Rb;  // full cost blocks [n_sub][nx][nx], [n_sub][nu][nu] (diag(q), diag(r) if none given)
  bool has_x = false, has_u = false, has_blk = false;
  int n_cx = 0, n_cu = 0;              // coupled rows per subsystem and slot kind
  std::vector<double> Gx, gx, Gu, gu;  // unit normals and right-hand sides
  double rho = 1, eps_p = 1e-4, eps_d = 1e-4;
  int max_iter = 1000;
  std::vector<std::vector<int32_t>> patch;  // local ids, ascending
  std::vector<std::vector<int32_t>> ring;
};

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// NVTX range over one entry point (visible to Nsight tools; free otherwise).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

}  // namespace

struct dlmpc_ctx {
  cudaStream_t stream = nullptr;
  int nx = 0, nu = 0, n_inst = 0, n_sub = 0;
  std::vector<Instance> inst;
  std::vector<Item> items;
  std::vector<int32_t> members, rev_slot, np_of;
  std::vector<int64_t> g_off;
  int64_t g_floats = 0, state_floats = 0;
  // reduced constraints
  std::vector<int64_t> zrow_ptr;
  std::vector<int32_t> zcol;
  std::vector<double> zval, rhs;
  std::vector<int64_t> rhs_off;
  std::vector<int32_t> kub;
  bool z_stale = false;  // the plant changed since the arrays above were built
  bool precomputed = false;
  int max_dcol = 0, max_kpad = 4, max_dred_pad = 4, max_nmem = 1;
  int64_t n_floats = 0, q_floats = 0;
  // launch plan of the sweep kernel
  int grid = 0, gt = 128, ng = 4, wave = 2, grp_floats = 0, cta_floats = 0, max_local_inst = 1;
  bool rows_cached = false;  // every group holds one wave: row records in shared memory
  size_t smem = 0;
  int64_t resident_n_items = 0, resident_state_items = 0;
  int residency = 2;  // 0: nothing resident, 1: compact iterate, Psi/Lambda and q resident, 2: also N
  int compact = 1;    // iterations after the first of a launch on the compact iterate
  bool block_cost = false;  // some instance has full cost blocks: slot box-QP Phi-step
  // Explicit solution of the slot QP with coupled rows (some instance has any):
  // per key 2 * global subsystem + kind (0 state, 1 input) the first region and
  // the region count, the first constraint row and the row count; per region
  // its active rows (count in bits 0..3, then 4 bits per row index).
  bool coupled = false;
  std::vector<int32_t> h_rg_base, h_rg_cnt, h_rw_base, h_rw_cnt;
  std::vector<uint32_t> h_rg_desc;
  std::vector<float> h_crow;  // rows: normal [nmax] then right-hand side
  int expl_stride = 0, crow_stride = 0;
  int force_block = 0;      // DLMPC_OPT_BLOCK_PHI
  unsigned long long stale_thr = 0, stale_seed = 0;  // DLMPC_OPT_STALE_PROB (floor(p 2^53)), _SEED
  int trace = 0;
  std::vector<int32_t> grp_ptr, grp_items, cta_inst_ptr, cta_inst;
  // options
  int fixed_iters = 0, max_iter_override = 0, export_phi = 0;
  double timeout_ms = 2000.0;
  std::string err;
  // device
  DevBuf<Item> d_items;
  DevBuf<int32_t> d_members, d_rev, d_np, d_grp_ptr, d_grp_items, d_cta_inst_ptr, d_cta_inst, d_adj_ptr, d_adj_idx,
      d_inst_iters, d_conv_prev, d_err, d_inst_item_ptr, d_sub_off;
  DevBuf<int64_t> d_goff;
  DevBuf<float> d_qblk2, d_rblk2, d_crow, d_expl;
  DevBuf<int32_t> d_rg_base, d_rg_cnt, d_rw_base, d_rw_cnt;
  DevBuf<uint32_t> d_rg_desc;
  DevBuf<float> d_N, d_q, d_cp, d_psi, d_lam, d_phi, d_G0, d_G1, d_S, d_qw, d_rw, d_xlo, d_xhi, d_ulo, d_uhi, d_rho,
      d_epsp, d_epsd, d_item_r, d_item_s, d_x, d_u, d_xn;
  DevBuf<double> d_Adiag, d_Aoff, d_B;
  DevBuf<unsigned long long> d_bar, d_trace;
  DevBuf<unsigned> d_notconv;
  DevBuf<dlmpc_stats> d_stats;
  DevBuf<const float *> d_ptr_in;
  DevBuf<float *> d_ptr_out, d_ptr_out2;
  dlmpc_stats *h_stats = nullptr;  // pinned
  int32_t *h_err = nullptr;        // pinned [8]
  int timing = 0;
  bool timed_step = false;
  bool kernel_events = false;
  int use_graph = 0;
  int plan_version = 0;
  struct GraphKey {
    const float *x;
    float *u, *xn;
    int warm;
    bool stats;
    int plan, fixed, max_iter;
    bool phi, trace;
    int compact, block;
    unsigned long long stale_thr, stale_seed;
    bool operator==(const GraphKey &o) const {
      return x == o.x && u == o.u && xn == o.xn && warm == o.warm && stats == o.stats && plan == o.plan &&
             fixed == o.fixed && max_iter == o.max_iter && phi == o.phi && trace == o.trace && compact == o.compact &&
             block == o.block && stale_thr == o.stale_thr && stale_seed == o.stale_seed;
    }
  };
  struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t capture_stream = nullptr;
  // learned warm start
  dlmpc_mlp *mlp = nullptr;
  int learn_L = 0, learn_slots = 1, learn_rsub = 1, learn_plant = 0;
  int skip_arrival_cta = -1;
  DevBuf<float> d_feat, d_lout, d_phi_l;
  // paper-variant ablation
  DevBuf<float> d_psi_prev;
  DevBuf<int32_t> d_row_sub, d_row_loc;
  float *h_exchange = nullptr;  // pinned, state_floats
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev_learn[2] = {nullptr, nullptr};

  ~dlmpc_ctx() {
    if (h_stats) cudaFreeHost(h_stats);
    if (h_err) cudaFreeHost(h_err);
    for (auto &e : ev)
      if (e) cudaEventDestroy(e);
    for (auto &e : ev_learn)
      if (e) cudaEventDestroy(e);
    for (auto &g : graphs) cudaGraphExecDestroy(g.exec);
    if (capture_stream) cudaStreamDestroy(capture_stream);
    if (h_exchange) cudaFreeHost(h_exchange);
  }
  int fail(int code, const std::string &msg) {
    err = msg;
    return code;
  }
  int cuda_fail(cudaError_t e, const char *what) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? DLMPC_ERR_NOMEM : DLMPC_ERR_CUDA;
  }
};

#define CK(call, what)                                      \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return ctx->cuda_fail(e_, what); \
  } while (0)

namespace {

template <class T>
cudaError_t upload(DevBuf<T> &b, const std::vector<T> &v, cudaStream_t s) {
  cudaError_t e = b.alloc(v.size());
  if (e != cudaSuccess || v.empty()) return e;
  return cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

// Hop distances from src up to max_hops (breadth-first search).
void bfs(const Instance &I, int src, int max_hops, std::vector<int> &dist, std::vector<int> &touched) {
  for (int v : touched) dist[v] = -1;
  touched.clear();
  std::vector<int> frontier{src};
  dist[src] = 0;
  touched.push_back(src);
  for (int h = 0; h < max_hops && !frontier.empty(); ++h) {
    std::vector<int> next;
    for (int v : frontier)
      for (int e = I.adj_ptr[v]; e < I.adj_ptr[v + 1]; ++e) {
        const int w = I.adj_idx[e];
        if (dist[w] < 0) {
          dist[w] = h + 1;
          touched.push_back(w);
          next.push_back(w);
        }
      }
    frontier.swap(next);
  }
}

// Rows A z <= b of the slot polytope of subsystem i (local index) for the
// slot kind (0: state slots t >= 1, 1: input slots): the finite box bounds as
// -z_a <= -lo_a, then z_a <= hi_a, then the coupled rows (unit normals).  The
// slot-0 state has no rows (Z_AB Psi = I pins it).
void slot_rows(const Instance &I, int nx, int nu, int i, int kind, std::vector<double> &A, std::vector<double> &b) {
  const int n = kind == 0 ? nx : nu;
  A.clear();
  b.clear();
  const bool box = kind == 0 ? I.has_x : I.has_u;
  const std::vector<double> &lo = kind == 0 ? I.x_lo : I.u_lo, &hi = kind == 0 ? I.x_hi : I.u_hi;
  if (box) {
    for (int side = 0; side < 2; ++side)
      for (int a = 0; a < n; ++a) {
        const double v = side == 0 ? lo[(size_t)i * n + a] : hi[(size_t)i * n + a];
        if (!std::isfinite(v)) continue;
        for (int c = 0; c < n; ++c) A.push_back(c == a ? (side == 0 ? -1.0 : 1.0) : 0.0);
        b.push_back(side == 0 ? -v : v);
      }
  }
  const int cnt = kind == 0 ? I.n_cx : I.n_cu;
  const std::vector<double> &G = kind == 0 ? I.Gx : I.Gu, &g = kind == 0 ? I.gx : I.gu;
  for (int k = 0; k < cnt; ++k) {
    for (int a = 0; a < n; ++a) A.push_back(G[((size_t)i * cnt + k) * n + a]);
    b.push_back(g[(size_t)i * cnt + k]);
  }
}

// Candidate active sets of the slot QP (the regions of its piecewise-affine
// explicit solution): every set of at most n rows with linearly independent
// normals (Cholesky of the Gram matrix), the empty set first.  Returns false
// when there are more than DLMPC_MAX_REGIONS.
bool slot_regions(const std::vector<double> &A, int m, int n, std::vector<uint32_t> &desc) {
  for (int k = 0; k <= std::min(n, m); ++k)
    for (uint32_t mask = 0; mask < (1u << m); ++mask) {
      if (__builtin_popcount(mask) != k) continue;
      int idx[kMaxNx] = {0}, c = 0;
      for (int r = 0; r < m; ++r)
        if (mask >> r & 1u) idx[c++] = r;
      double L[kMaxNx * kMaxNx] = {0};
      bool indep = true;
      for (int a = 0; a < k && indep; ++a)
        for (int e = 0; e <= a; ++e) {
          double v = 0;
          for (int t = 0; t < n; ++t) v += A[(size_t)idx[a] * n + t] * A[(size_t)idx[e] * n + t];
          for (int t = 0; t < e; ++t) v -= L[a * kMaxNx + t] * L[e * kMaxNx + t];
          if (a == e) {
            if (!(v > 1e-10)) { indep = false; break; }
            L[a * kMaxNx + a] = std::sqrt(v);
          } else {
            L[a * kMaxNx + e] = v / L[e * kMaxNx + e];
          }
        }
      if (!indep) continue;
      uint32_t d = (uint32_t)k;
      for (int a = 0; a < k; ++a) d |= (uint32_t)idx[a] << (4 + 4 * a);
      desc.push_back(d);
      if ((int)desc.size() > DLMPC_MAX_REGIONS) return false;
    }
  return true;
}

int validate(const dlmpc_problem &p, int nx, int nu, std::string &msg) {
  char buf[256];
  if (p.n_sub < 1 || p.nx < 1 || p.nu < 1 || p.nx > kMaxNx || p.nu > kMaxNu || p.T < 2 || p.d < 0) {
    snprintf(buf, sizeof buf, "bad sizes n_sub=%d nx=%d nu=%d T=%d d=%d", p.n_sub, p.nx, p.nu, p.T, p.d);
    msg = buf;
    return DLMPC_ERR_ARG;
  }
  if (p.nx != nx || p.nu != nu) { msg = "all instances must share nx and nu"; return DLMPC_ERR_ARG; }
  if (!p.adj_ptr || !p.A_diag || !p.B || !p.q || !p.r) { msg = "missing required array"; return DLMPC_ERR_ARG; }
  if (p.adj_ptr[0] != 0) { msg = "adj_ptr[0] must be 0"; return DLMPC_ERR_ARG; }
  const int nnz = p.adj_ptr[p.n_sub];
  if (nnz > 0 && (!p.adj_idx || !p.A_off)) { msg = "missing adjacency arrays"; return DLMPC_ERR_ARG; }
  for (int i = 0; i < p.n_sub; ++i) {
    if (p.adj_ptr[i + 1] < p.adj_ptr[i]) { msg = "adj_ptr not monotone"; return DLMPC_ERR_ARG; }
    for (int e = p.adj_ptr[i]; e < p.adj_ptr[i + 1]; ++e)
      if (p.adj_idx[e] < 0 || p.adj_idx[e] >= p.n_sub || p.adj_idx[e] == i) {
        msg = "adj_idx out of range or self loop";
        return DLMPC_ERR_ARG;
      }
  }
  if (!(p.rho > 0) || !(p.eps_p > 0) || !(p.eps_d > 0) || p.max_iter < 1) {
    msg = "rho, eps_p, eps_d must be > 0 and max_iter >= 1";
    return DLMPC_ERR_ARG;
  }
  for (int i = 0; i < p.n_sub * nx; ++i)
    if (!(p.q[i] >= 0)) { msg = "q must be >= 0"; return DLMPC_ERR_ARG; }
  for (int i = 0; i < p.n_sub * nu; ++i)
    if (!(p.r[i] >= 0)) { msg = "r must be >= 0"; return DLMPC_ERR_ARG; }
  if ((p.x_lo == nullptr) != (p.x_hi == nullptr) || (p.u_lo == nullptr) != (p.u_hi == nullptr)) {
    msg = "bounds must be given in lo/hi pairs";
    return DLMPC_ERR_ARG;
  }
  if (p.u_lo)
    for (int i = 0; i < p.n_sub * nu; ++i)
      if (!(p.u_lo[i] <= 0 && p.u_hi[i] >= 0)) { msg = "0 must lie in [u_lo, u_hi]"; return DLMPC_ERR_ARG; }
  if (p.x_lo)
    for (int i = 0; i < p.n_sub * nx; ++i)
      if (!(p.x_lo[i] <= 0 && p.x_hi[i] >= 0)) { msg = "0 must lie in [x_lo, x_hi]"; return DLMPC_ERR_ARG; }
  // coupled rows: counts in range, nonzero finite normals, g >= 0 (0 feasible)
  if (p.n_cx < 0 || p.n_cx > DLMPC_MAX_COUPLED || p.n_cu < 0 || p.n_cu > DLMPC_MAX_COUPLED) {
    msg = "n_cx and n_cu must lie in 0..DLMPC_MAX_COUPLED";
    return DLMPC_ERR_ARG;
  }
  for (int kind = 0; kind < 2; ++kind) {
    const int cnt = kind == 0 ? p.n_cx : p.n_cu, n = kind == 0 ? nx : nu;
    const double *G = kind == 0 ? p.Gx : p.Gu, *g = kind == 0 ? p.gx : p.gu;
    if (cnt == 0) continue;
    if (!G || !g) { msg = "Gx/gx (Gu/gu) must be given when n_cx (n_cu) > 0"; return DLMPC_ERR_ARG; }
    for (int e = 0; e < p.n_sub * cnt; ++e) {
      double nrm = 0;
      for (int a = 0; a < n; ++a) nrm += G[(size_t)e * n + a] * G[(size_t)e * n + a];
      if (!(nrm > 0) || !std::isfinite(nrm)) { msg = "coupled rows need finite nonzero normals"; return DLMPC_ERR_ARG; }
      if (!(g[e] >= 0) || !std::isfinite(g[e])) { msg = "coupled right-hand sides must be finite and >= 0"; return DLMPC_ERR_ARG; }
    }
  }
  // full cost blocks: symmetric and positive definite (Cholesky must succeed)
  for (int which = 0; which < 2; ++which) {
    const double *blk = which == 0 ? p.Q_blk : p.R_blk;
    const int n = which == 0 ? nx : nu;
    if (!blk) continue;
    for (int i = 0; i < p.n_sub; ++i) {
      const double *M = blk + (size_t)i * n * n;
      double L[kMaxNx * kMaxNx] = {0};
      for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
          if (!(std::fabs(M[a * n + b] - M[b * n + a]) <= 1e-12 * (1.0 + std::fabs(M[a * n + b])))) {
            msg = "Q_blk / R_blk must be symmetric";
            return DLMPC_ERR_ARG;
          }
        }
      for (int a = 0; a < n; ++a)
        for (int b = 0; b <= a; ++b) {
          double v = M[a * n + b];
          for (int c = 0; c < b; ++c) v -= L[a * n + c] * L[b * n + c];
          if (a == b) {
            if (!(v > 0)) { msg = "Q_blk / R_blk must be positive definite"; return DLMPC_ERR_ARG; }
            L[a * n + a] = std::sqrt(v);
          } else {
            L[a * n + b] = v / L[b * n + b];
          }
        }
    }
  }
  return 0;
}

// Restricted constraint of column patch j in the reduced variables (slot-0
// states of the patch are fixed to e_c and moved to the right-hand side).
// Appends CSR rows and nx right-hand sides; returns rows kept, or -1 if a row
// without patch variables has a nonzero right-hand side (locality infeasible).
int build_reduced(const Instance &I, int nx, int nu, int j, std::vector<int64_t> &rptr, std::vector<int32_t> &col,
                  std::vector<double> &val, std::vector<double> &rhs_out) {
  const auto &patch = I.patch[j];
  const auto &ring = I.ring[j];
  const int T = I.T;
  const int r_sub = nx * T + nu * (T - 1);
  const int rsr = r_sub - nx;
  auto pos_of = [&](int i) -> int {
    auto it = std::lower_bound(patch.begin(), patch.end(), i);
    return (it != patch.end() && *it == i) ? int(it - patch.begin()) : -1;
  };
  std::vector<std::vector<double>> rhs_rows;  // per kept row: nx values
  std::vector<std::pair<int32_t, double>> ent;
  for (int t = 1; t < T; ++t)
    for (int i : ring) {
      const int pi = pos_of(i);
      for (int a = 0; a < nx; ++a) {
        ent.clear();
        std::vector<double> b(nx, 0.0);
        auto add_state = [&](int k, int pk, int slot, int bb, double coef) {
          if (coef == 0.0 || pk < 0) return;
          if (slot == 0) {
            // x_0 of patch member k is e_c: moves to the right-hand side
            if (k == j) b[bb] -= coef;
          } else {
            ent.emplace_back(pk * rsr + slot * nx + bb - nx, coef);
          }
        };
        add_state(i, pi, t, a, 1.0);
        for (int bb = 0; bb < nx; ++bb) add_state(i, pi, t - 1, bb, -I.A_diag[((size_t)i * nx + a) * nx + bb]);
        for (int e = I.adj_ptr[i]; e < I.adj_ptr[i + 1]; ++e) {
          const int k = I.adj_idx[e];
          const int pk = pos_of(k);
          for (int bb = 0; bb < nx; ++bb) add_state(k, pk, t - 1, bb, -I.A_off[((size_t)e * nx + a) * nx + bb]);
        }
        if (pi >= 0)
          for (int e = 0; e < nu; ++e) {
            const double coef = -I.B[((size_t)i * nx + a) * nu + e];
            if (coef != 0.0) ent.emplace_back(pi * rsr + nx * (T - 1) + (t - 1) * nu + e, coef);
          }
        if (ent.empty()) {
          for (double v : b)
            if (v != 0.0) return -1;
          continue;
        }
        std::sort(ent.begin(), ent.end());
        // merge duplicates
        std::vector<std::pair<int32_t, double>> merged;
        for (auto &pr : ent) {
          if (!merged.empty() && merged.back().first == pr.first) merged.back().second += pr.second;
          else merged.push_back(pr);
        }
        for (auto &pr : merged) {
          col.push_back(pr.first);
          val.push_back(pr.second);
        }
        rptr.push_back((int64_t)col.size());
        rhs_rows.push_back(b);
      }
    }
  const int m = (int)rhs_rows.size();
  for (int c = 0; c < nx; ++c)
    for (int row = 0; row < m; ++row) rhs_out.push_back(rhs_rows[row][c]);
  return m;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" int dlmpc_setup(const dlmpc_problem *probs, int32_t n_inst, void *stream, dlmpc_ctx **out) {
  NvtxRange range("dlmpc_setup");
  g_setup_error.clear();
  if (!out || !probs || n_inst < 1) {
    g_setup_error = "dlmpc_setup: null argument or n_inst < 1";
    return DLMPC_ERR_ARG;
  }
  *out = nullptr;
  auto *ctx = new (std::nothrow) dlmpc_ctx();
  if (!ctx) return DLMPC_ERR_NOMEM;
  ctx->stream = static_cast<cudaStream_t>(stream);
  ctx->nx = probs[0].nx;
  ctx->nu = probs[0].nu;
  ctx->n_inst = n_inst;
  const int nx = ctx->nx, nu = ctx->nu;
  for (int b = 0; b < n_inst; ++b) {
    std::string msg;
    int rc = validate(probs[b], nx, nu, msg);
    if (rc) {
      g_setup_error = "instance " + std::to_string(b) + ": " + msg;
      delete ctx;
      return rc;
    }
  }
  ctx->inst.resize(n_inst);
  int sub_off = 0;
  for (int b = 0; b < n_inst; ++b) {
    const dlmpc_problem &p = probs[b];
    Instance &I = ctx->inst[b];
    I.n_sub = p.n_sub;
    I.T = p.T;
    I.d = p.d;
    I.sub_off = sub_off;
    I.item_off = sub_off;
    sub_off += p.n_sub;
    const int nnz = p.adj_ptr[p.n_sub];
    I.adj_ptr.assign(p.adj_ptr, p.adj_ptr + p.n_sub + 1);
    I.adj_idx.assign(p.adj_idx, p.adj_idx + nnz);
    I.A_diag.assign(p.A_diag, p.A_diag + (size_t)p.n_sub * nx * nx);
    I.A_off.assign(p.A_off, p.A_off + (size_t)nnz * nx * nx);
    I.B.assign(p.B, p.B + (size_t)p.n_sub * nx * nu);
    I.q.assign(p.q, p.q + (size_t)p.n_sub * nx);
    I.r.assign(p.r, p.r + (size_t)p.n_sub * nu);
    I.has_blk = p.Q_blk != nullptr || p.R_blk != nullptr;
    I.Qb.assign((size_t)p.n_sub * nx * nx, 0.0);
    I.Rb.assign((size_t)p.n_sub * nu * nu, 0.0);
    for (int i = 0; i < p.n_sub; ++i) {
      for (int a = 0; a < nx; ++a)
        for (int b = 0; b < nx; ++b)
          I.Qb[((size_t)i * nx + a) * nx + b] =
              p.Q_blk ? p.Q_blk[((size_t)i * nx + a) * nx + b] : (a == b ? p.q[(size_t)i * nx + a] : 0.0);
      for (int a = 0; a < nu; ++a)
        for (int b = 0; b < nu; ++b)
          I.Rb[((size_t)i * nu + a) * nu + b] =
              p.R_blk ? p.R_blk[((size_t)i * nu + a) * nu + b] : (a == b ? p.r[(size_t)i * nu + a] : 0.0);
    }
    I.n_cx = p.n_cx;
    I.n_cu = p.n_cu;
    for (int kind = 0; kind < 2; ++kind) {
      const int cnt = kind == 0 ? p.n_cx : p.n_cu, n = kind == 0 ? nx : nu;
      const double *G = kind == 0 ? p.Gx : p.Gu, *g = kind == 0 ? p.gx : p.gu;
      std::vector<double> &Go = kind == 0 ? I.Gx : I.Gu, &go = kind == 0 ? I.gx : I.gu;
      for (int e = 0; e < p.n_sub * cnt; ++e) {
        double nrm = 0;
        for (int a = 0; a < n; ++a) nrm += G[(size_t)e * n + a] * G[(size_t)e * n + a];
        nrm = std::sqrt(nrm);
        for (int a = 0; a < n; ++a) Go.push_back(G[(size_t)e * n + a] / nrm);
        go.push_back(g[e] / nrm);
      }
    }
    I.has_x = p.x_lo != nullptr;
    I.has_u = p.u_lo != nullptr;
    if (I.has_x) {
      I.x_lo.assign(p.x_lo, p.x_lo + (size_t)p.n_sub * nx);
      I.x_hi.assign(p.x_hi, p.x_hi + (size_t)p.n_sub * nx);
    }
    if (I.has_u) {
      I.u_lo.assign(p.u_lo, p.u_lo + (size_t)p.n_sub * nu);
      I.u_hi.assign(p.u_hi, p.u_hi + (size_t)p.n_sub * nu);
    }
    I.rho = p.rho;
    I.eps_p = p.eps_p;
    I.eps_d = p.eps_d;
    I.max_iter = p.max_iter;
    // d-hop patches and (d+1)-hop rings
    std::vector<int> dist(p.n_sub, -1), touched;
    I.patch.resize(p.n_sub);
    I.ring.resize(p.n_sub);
    for (int i = 0; i < p.n_sub; ++i) {
      bfs(I, i, p.d + 1, dist, touched);
      for (int v : touched) {
        if (dist[v] <= p.d) I.patch[i].push_back(v);
        I.ring[i].push_back(v);
      }
      std::sort(I.patch[i].begin(), I.patch[i].end());
      std::sort(I.ring[i].begin(), I.ring[i].end());
    }
  }
  ctx->n_sub = sub_off;
  // items, exchange layout, reduced constraints
  ctx->items.resize(ctx->n_sub);
  ctx->np_of.resize(ctx->n_sub);
  ctx->g_off.resize(ctx->n_sub);
  int64_t goff = 0, st_off = 0, q_off = 0;
  for (int b = 0; b < n_inst; ++b) {
    const Instance &I = ctx->inst[b];
    const int r_sub = nx * I.T + nu * (I.T - 1);
    for (int i = 0; i < I.n_sub; ++i) {
      const int g = I.sub_off + i;
      ctx->np_of[g] = (int)I.patch[i].size();
      ctx->g_off[g] = goff;
      goff += (int64_t)ctx->np_of[g] * r_sub;
    }
  }
  ctx->g_floats = goff;
  ctx->zrow_ptr.clear();
  ctx->kub.resize(ctx->n_sub);
  ctx->rhs_off.resize(ctx->n_sub);
  for (int b = 0; b < n_inst; ++b) {
    const Instance &I = ctx->inst[b];
    const int r_sub = nx * I.T + nu * (I.T - 1);
    for (int j = 0; j < I.n_sub; ++j) {
      const int g = I.sub_off + j;
      Item &it = ctx->items[g];
      it.inst = b;
      it.sub = g;
      it.n_mem = (int)I.patch[j].size();
      it.mem_off = (int)ctx->members.size();
      it.self_pos = int(std::lower_bound(I.patch[j].begin(), I.patch[j].end(), j) - I.patch[j].begin());
      it.r_sub = r_sub;
      it.T = I.T;
      it.dred = (r_sub - nx) * it.n_mem;
      it.dred_pad = (int)round_up(it.dred, 4);
      it.st_off = st_off;
      st_off += (int64_t)nx * r_sub * it.n_mem;
      it.q_off = q_off;
      q_off += (int64_t)nx * it.dred_pad;
      for (int m : I.patch[j]) {
        ctx->members.push_back(I.sub_off + m);
        const auto &pm = I.patch[m];
        ctx->rev_slot.push_back(int(std::lower_bound(pm.begin(), pm.end(), j) - pm.begin()));
      }
      it.z_off = (int64_t)ctx->zrow_ptr.size();
      ctx->zrow_ptr.push_back((int64_t)ctx->zcol.size());
      ctx->rhs_off[g] = (int64_t)ctx->rhs.size();
      const int m = build_reduced(I, nx, nu, j, ctx->zrow_ptr, ctx->zcol, ctx->zval, ctx->rhs);
      if (m < 0) {
        g_setup_error = "instance " + std::to_string(b) + " subsystem " + std::to_string(j) +
                        ": locality constraint infeasible (row without patch variables has nonzero RHS)";
        delete ctx;
        return DLMPC_ERR_INFEASIBLE_LOCALITY;
      }
      it.mrows = m;
      ctx->kub[g] = std::max(1, nu * (I.T - 1) * it.n_mem);
      it.k = 0;
      it.kpad = 1;
      ctx->max_dcol = std::max(ctx->max_dcol, r_sub * it.n_mem);
      ctx->max_nmem = std::max(ctx->max_nmem, it.n_mem);
    }
  }
  ctx->state_floats = st_off;
  ctx->q_floats = q_off;
  // regions of the explicit slot-QP solution when some instance has coupled rows
  for (const Instance &I : ctx->inst) ctx->coupled = ctx->coupled || I.n_cx > 0 || I.n_cu > 0;
  if (ctx->coupled) {
    const int nmax = std::max(nx, nu);
    ctx->expl_stride = 2 * (nmax * nmax + nmax);  // K, k, L, l
    ctx->crow_stride = nmax + 1;
    std::vector<double> A, bb;
    for (const Instance &I : ctx->inst)
      for (int i = 0; i < I.n_sub; ++i)
        for (int kind = 0; kind < 2; ++kind) {
          const int n = kind == 0 ? nx : nu;
          slot_rows(I, nx, nu, i, kind, A, bb);
          const int m = (int)bb.size();
          ctx->h_rw_base.push_back((int32_t)(ctx->h_crow.size() / ctx->crow_stride));
          ctx->h_rw_cnt.push_back(m);
          for (int r = 0; r < m; ++r) {
            for (int a = 0; a < nmax; ++a) ctx->h_crow.push_back(a < n ? (float)A[(size_t)r * n + a] : 0.f);
            ctx->h_crow.push_back((float)bb[r]);
          }
          std::vector<uint32_t> desc;
          if (!slot_regions(A, m, n, desc)) {
            g_setup_error = "a slot has more than DLMPC_MAX_REGIONS candidate active sets";
            delete ctx;
            return DLMPC_ERR_ARG;
          }
          ctx->h_rg_base.push_back((int32_t)ctx->h_rg_desc.size());
          ctx->h_rg_cnt.push_back((int32_t)desc.size());
          ctx->h_rg_desc.insert(ctx->h_rg_desc.end(), desc.begin(), desc.end());
        }
  }
  *out = ctx;
  return DLMPC_OK;
}

namespace {

int upload_static(dlmpc_ctx *ctx) {
  const int nx = ctx->nx, nu = ctx->nu;
  cudaStream_t s = ctx->stream;
  std::vector<float> qw, rw, xlo, xhi, ulo, uhi, rho, epsp, epsd, qblk2, rblk2;
  std::vector<double> Ad, Ao, Bm;
  std::vector<int32_t> aptr{0}, aidx, inst_item_ptr{0};
  for (const Instance &I : ctx->inst) {
    const float inf = std::numeric_limits<float>::infinity();
    for (int i = 0; i < I.n_sub; ++i) {
      for (int a = 0; a < nx; ++a) {
        qw.push_back((float)I.q[(size_t)i * nx + a]);
        xlo.push_back(I.has_x ? (float)I.x_lo[(size_t)i * nx + a] : -inf);
        xhi.push_back(I.has_x ? (float)I.x_hi[(size_t)i * nx + a] : inf);
      }
      for (int e = 0; e < nu; ++e) {
        rw.push_back((float)I.r[(size_t)i * nu + e]);
        ulo.push_back(I.has_u ? (float)I.u_lo[(size_t)i * nu + e] : -inf);
        uhi.push_back(I.has_u ? (float)I.u_hi[(size_t)i * nu + e] : inf);
      }
      for (int e = I.adj_ptr[i]; e < I.adj_ptr[i + 1]; ++e) aidx.push_back(I.sub_off + I.adj_idx[e]);
      aptr.push_back((int32_t)aidx.size());
    }
    for (double v : I.Qb) qblk2.push_back((float)(2.0 * v));
    for (double v : I.Rb) rblk2.push_back((float)(2.0 * v));
    ctx->block_cost = ctx->block_cost || I.has_blk || I.n_cx > 0 || I.n_cu > 0;
    Ad.insert(Ad.end(), I.A_diag.begin(), I.A_diag.end());
    Ao.insert(Ao.end(), I.A_off.begin(), I.A_off.end());
    Bm.insert(Bm.end(), I.B.begin(), I.B.end());
    rho.push_back((float)I.rho);
    epsp.push_back((float)I.eps_p);
    epsd.push_back((float)I.eps_d);
    inst_item_ptr.push_back(I.item_off + I.n_sub);
  }
  CK(upload(ctx->d_qw, qw, s), "upload qw");
  CK(upload(ctx->d_qblk2, qblk2, s), "upload Q blocks");
  CK(upload(ctx->d_rblk2, rblk2, s), "upload R blocks");
  if (ctx->coupled) {
    CK(upload(ctx->d_rg_base, ctx->h_rg_base, s), "upload regions");
    CK(upload(ctx->d_rg_cnt, ctx->h_rg_cnt, s), "upload regions");
    CK(upload(ctx->d_rw_base, ctx->h_rw_base, s), "upload rows");
    CK(upload(ctx->d_rw_cnt, ctx->h_rw_cnt, s), "upload rows");
    CK(upload(ctx->d_rg_desc, ctx->h_rg_desc, s), "upload regions");
    CK(upload(ctx->d_crow, ctx->h_crow, s), "upload rows");
    CK(ctx->d_expl.alloc((size_t)ctx->h_rg_desc.size() * ctx->expl_stride), "alloc explicit solution");
  }
  CK(upload(ctx->d_rw, rw, s), "upload rw");
  CK(upload(ctx->d_xlo, xlo, s), "upload xlo");
  CK(upload(ctx->d_xhi, xhi, s), "upload xhi");
  CK(upload(ctx->d_ulo, ulo, s), "upload ulo");
  CK(upload(ctx->d_uhi, uhi, s), "upload uhi");
  CK(upload(ctx->d_rho, rho, s), "upload rho");
  CK(upload(ctx->d_epsp, epsp, s), "upload eps");
  CK(upload(ctx->d_epsd, epsd, s), "upload eps");
  CK(upload(ctx->d_Adiag, Ad, s), "upload A");
  CK(upload(ctx->d_Aoff, Ao, s), "upload A");
  CK(upload(ctx->d_B, Bm, s), "upload B");
  CK(upload(ctx->d_adj_ptr, aptr, s), "upload adjacency");
  CK(upload(ctx->d_adj_idx, aidx, s), "upload adjacency");
  CK(upload(ctx->d_inst_item_ptr, inst_item_ptr, s), "upload instance offsets");
  CK(upload(ctx->d_members, ctx->members, s), "upload members");
  CK(upload(ctx->d_rev, ctx->rev_slot, s), "upload rev");
  CK(upload(ctx->d_np, ctx->np_of, s), "upload np");
  CK(upload(ctx->d_goff, ctx->g_off, s), "upload goff");
  std::vector<int32_t> sub_off;
  for (const Instance &I : ctx->inst) sub_off.push_back(I.sub_off);
  sub_off.push_back(ctx->n_sub);
  CK(upload(ctx->d_sub_off, sub_off, s), "upload sub offsets");
  CK(ctx->d_psi.alloc(ctx->state_floats), "alloc Psi");
  CK(ctx->d_lam.alloc(ctx->state_floats), "alloc Lambda");
  CK(cudaMemsetAsync(ctx->d_psi.p, 0, ctx->state_floats * 4, s), "memset");
  CK(cudaMemsetAsync(ctx->d_lam.p, 0, ctx->state_floats * 4, s), "memset");
  CK(ctx->d_G0.alloc(ctx->g_floats), "alloc exchange");
  CK(ctx->d_G1.alloc(ctx->g_floats), "alloc exchange");
  CK(ctx->d_S.alloc(ctx->n_sub), "alloc S");
  CK(ctx->d_item_r.alloc(ctx->n_sub), "alloc residuals");
  CK(ctx->d_item_s.alloc(ctx->n_sub), "alloc residuals");
  CK(ctx->d_bar.alloc(3), "alloc barrier");
  CK(ctx->d_notconv.alloc(3 * ctx->n_inst), "alloc conv");
  CK(ctx->d_inst_iters.alloc(ctx->n_inst), "alloc iters");
  CK(ctx->d_conv_prev.alloc(ctx->n_inst), "alloc conv flags");
  CK(cudaMemsetAsync(ctx->d_conv_prev.p, 0, sizeof(int32_t) * ctx->n_inst, s), "memset");
  CK(ctx->d_err.alloc(8), "alloc err");
  CK(ctx->d_stats.alloc(ctx->n_inst), "alloc stats");
  CK(ctx->d_x.alloc((size_t)ctx->n_sub * nx), "alloc staging");
  CK(ctx->d_u.alloc((size_t)ctx->n_sub * nu), "alloc staging");
  CK(ctx->d_xn.alloc((size_t)ctx->n_sub * nx), "alloc staging");
  CK(cudaMallocHost(&ctx->h_stats, sizeof(dlmpc_stats) * ctx->n_inst), "alloc pinned");
  CK(cudaMallocHost(&ctx->h_err, sizeof(int32_t) * 8), "alloc pinned");
  return 0;
}

double item_cost(const dlmpc_ctx *ctx, const Item &it) {
  return (double)it.dred * (2.0 * it.k + 4.0 * ctx->nx) + 8.0 * it.r_sub * it.n_mem + 2000.0;
}

// Longest-processing-time assignment of `ids` to `bins` bins.
std::vector<std::vector<int32_t>> lpt(const dlmpc_ctx *ctx, const std::vector<int32_t> &ids, int bins) {
  std::vector<int32_t> order = ids;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return item_cost(ctx, ctx->items[a]) > item_cost(ctx, ctx->items[b]);
  });
  using P = std::pair<double, int>;
  std::priority_queue<P, std::vector<P>, std::greater<P>> heap;
  for (int b = 0; b < bins; ++b) heap.push({0.0, b});
  std::vector<std::vector<int32_t>> out(bins);
  for (int g : order) {
    auto top = heap.top();
    heap.pop();
    out[top.second].push_back(g);
    heap.push({top.first + item_cost(ctx, ctx->items[g]), top.second});
  }
  return out;
}

// Plans the sweep launch for `gt` threads per group, `ng` groups per CTA and
// Phi-step waves of `wave` items: one CTA per SM, items assigned to CTAs and
// groups by longest processing time, then each CTA's shared-memory arena
// filled with resident Psi/Lambda and q, then resident N, until it is full.
int plan_sweep(dlmpc_ctx *ctx, int gt, int ng, int wave, bool exact_groups = false) {
  // named barrier ids 1..15 serve the groups (id 0 is __syncthreads)
  if (!(gt == 64 || gt == 96 || gt == 128 || gt == 256) || ng < 1 || ng > 15 || gt * ng > 1024 || wave < 1 || wave > 8)
    return ctx->fail(DLMPC_ERR_ARG, "unsupported sweep shape");
  if (ctx->max_kpad > 4 * gt) return ctx->fail(DLMPC_ERR_ARG, "null-space dimension too large for this group size");
  const int nx = ctx->nx;
  int dev = 0, sms = 0, smem_optin = 0;
  CK(cudaGetDevice(&dev), "cudaGetDevice");
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "attr");
  CK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "attr");
  const int n = ctx->n_sub;
  // default: every SM busy, groups per CTA trimmed to the items per CTA;
  // an explicit shape keeps its group count and trims the grid instead
  const int grid = exact_groups ? std::max(1, std::min(sms, (n + ng - 1) / ng)) : std::max(1, std::min(sms, n));
  if (!exact_groups) ng = std::max(1, std::min(ng, (n + grid - 1) / grid));
  // the kernel of the final CTA size (its register tier)
  const void *fn = sweep_kernel_ptr(nx, gt, false, gt * ng);
  if (!fn) return ctx->fail(DLMPC_ERR_ARG, "no sweep kernel for this nx / group size");
  const void *fn_blk = sweep_kernel_ptr(nx, gt, true, gt * ng);  // full cost blocks (64 and 128 threads)
  if (ctx->block_cost && !fn_blk)
    return ctx->fail(DLMPC_ERR_ARG, "full cost blocks need 64 or 128 threads per group");
  cudaFuncAttributes fa{};
  CK(cudaFuncGetAttributes(&fa, fn), "cudaFuncGetAttributes");
  const int64_t budget = ((int64_t)smem_optin - (int64_t)fa.sharedSizeBytes - 64) / 4;  // floats
  std::vector<int32_t> all(n);
  std::iota(all.begin(), all.end(), 0);
  auto ctas = lpt(ctx, all, grid);
  int max_li = 1;
  for (auto &ci : ctas) {
    std::vector<int> insts;
    for (int g : ci) insts.push_back(ctx->items[g].inst);
    std::sort(insts.begin(), insts.end());
    insts.erase(std::unique(insts.begin(), insts.end()), insts.end());
    max_li = std::max<int>(max_li, (int)insts.size());
  }
  const int cta_floats = 8 + 4 * ((3 * max_li + 3) / 4);
  int64_t used_max = 0;
  std::vector<std::vector<std::vector<int32_t>>> groups(grid);
  // groups of one wave keep their patch rows' records in shared memory
  // (filled once per launch); otherwise the records are derived in the loop
  bool rows_cached = true;
  for (int b = 0; b < grid; ++b) {
    groups[b] = lpt(ctx, ctas[b], ng);
    for (auto &gl : groups[b]) rows_cached = rows_cached && (int)gl.size() <= wave;
  }
  {  // N that is not resident is read from global memory directly
    const int grp = sweep_group_floats(nx, ctx->nu, gt, wave, ctx->max_dcol, ctx->max_dred_pad, ctx->max_kpad,
                                       ctx->max_nmem, rows_cached);
    const int64_t arena_cap = budget - (int64_t)ng * grp - cta_floats;
    if (arena_cap < 0) return ctx->fail(DLMPC_ERR_ARG, "shared-memory budget exceeded by the group buffers");
    used_max = 0;
    ctx->resident_n_items = ctx->resident_state_items = 0;
    for (int b = 0; b < grid; ++b) {
      int64_t used = 0;
      // resident Psi/Lambda and q first (round robin over groups)
      std::vector<int32_t> rr;
      size_t depth = 0;
      for (bool more = true; more; ++depth) {
        more = false;
        for (auto &gl : groups[b])
          if (depth < gl.size()) { rr.push_back(gl[depth]); more = true; }
      }
      // the compact iterate (touched every iteration), then N (read twice per
      // iteration), then Psi/Lambda and q (first iteration and the ends of
      // a launch, or every iteration when Phi is exported)
      for (int id : rr) {
        Item &it = ctx->items[id];
        const int64_t need = cp_floats(it, nx);
        it.n_sm = it.q_sm = it.st_sm = it.cp_sm = -1;
        if (ctx->residency >= 1 && used + need <= arena_cap) {
          it.cp_sm = (int32_t)used;
          used += need;
        }
      }
      for (int id : rr) {
        Item &it = ctx->items[id];
        const int64_t need = (int64_t)it.dred_pad * it.kpad;  // N only: resident patches skip N^T
        if (ctx->residency >= 2 && used + need <= arena_cap) {
          it.n_sm = (int32_t)used;
          used += need;
          ++ctx->resident_n_items;
        }
      }
      for (int id : rr) {
        Item &it = ctx->items[id];
        const int64_t need = 2LL * nx * it.r_sub * it.n_mem + (int64_t)nx * it.dred_pad;
        if (ctx->residency >= 1 && used + need <= arena_cap) {
          it.st_sm = (int32_t)used;
          it.q_sm = (int32_t)(used + 2LL * nx * it.r_sub * it.n_mem);
          used += need;
          ++ctx->resident_state_items;
        }
      }
      used_max = std::max(used_max, used);
      // resident-N items first within each group
      for (auto &gl : groups[b])
        std::stable_partition(gl.begin(), gl.end(), [&](int id) { return ctx->items[id].n_sm >= 0; });
    }
    ctx->grp_floats = grp;
    ctx->rows_cached = rows_cached;
  }
  ctx->grid = grid;
  ctx->gt = gt;
  ctx->ng = ng;
  ctx->wave = wave;
  ctx->cta_floats = cta_floats;
  ctx->max_local_inst = max_li;
  ctx->grp_ptr.assign(1, 0);
  ctx->grp_items.clear();
  ctx->cta_inst_ptr.assign(1, 0);
  ctx->cta_inst.clear();
  for (int b = 0; b < grid; ++b) {
    std::vector<int> insts;
    for (int g : ctas[b]) insts.push_back(ctx->items[g].inst);
    std::sort(insts.begin(), insts.end());
    insts.erase(std::unique(insts.begin(), insts.end()), insts.end());
    for (int g : ctas[b])
      ctx->items[g].lslot = int(std::lower_bound(insts.begin(), insts.end(), ctx->items[g].inst) - insts.begin());
    ctx->cta_inst.insert(ctx->cta_inst.end(), insts.begin(), insts.end());
    ctx->cta_inst_ptr.push_back((int32_t)ctx->cta_inst.size());
    for (auto &gl : groups[b]) {
      ctx->grp_items.insert(ctx->grp_items.end(), gl.begin(), gl.end());
      ctx->grp_ptr.push_back((int32_t)ctx->grp_items.size());
    }
  }
  ctx->smem = (size_t)((int64_t)ng * ctx->grp_floats + cta_floats + used_max) * 4;
  ++ctx->plan_version;
  CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ctx->smem), "smem attr");
  if (fn_blk) CK(cudaFuncSetAttribute(fn_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ctx->smem), "smem attr");
  int occ = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, gt * ng, ctx->smem), "occupancy");
  if (occ < 1 || grid > occ * sms) return ctx->fail(DLMPC_ERR_ARG, "sweep kernel cannot be co-resident");
  cudaStream_t s = ctx->stream;
  CK(upload(ctx->d_items, ctx->items, s), "upload items");
  CK(upload(ctx->d_grp_ptr, ctx->grp_ptr, s), "upload plan");
  CK(upload(ctx->d_grp_items, ctx->grp_items, s), "upload plan");
  CK(upload(ctx->d_cta_inst_ptr, ctx->cta_inst_ptr, s), "upload plan");
  CK(upload(ctx->d_cta_inst, ctx->cta_inst, s), "upload plan");
  return 0;
}

}  // namespace

namespace {

// Packed operator layout from the null-space dimensions: odd row stride kpad,
// 16-byte aligned items (N then N^T), compact iterates; allocates N (not
// filled) and the compact iterates and uploads the items.
int operator_layout(dlmpc_ctx *ctx, const std::vector<int32_t> &nul) {
  cudaStream_t s = ctx->stream;
  int64_t noff = 0;
  ctx->max_kpad = 1;
  for (int g = 0; g < ctx->n_sub; ++g) {
    Item &it = ctx->items[g];
    it.k = nul[g];
    // row stride: multiple of 4 floats (16-byte vector loads) with an odd
    // number of 16-byte units, so consecutive rows hit distinct bank groups
    it.kpad = (int)round_up(std::max(it.k, 1), 4);
    if ((it.kpad / 4) % 2 == 0) it.kpad += 4;
    it.n_off = noff;
    noff += round_up((int64_t)n_floats(it), 4);
    ctx->max_kpad = std::max(ctx->max_kpad, it.kpad);
    ctx->max_dred_pad = std::max(ctx->max_dred_pad, it.dred_pad);
  }
  ctx->n_floats = noff;
  int64_t cpoff = 0;
  for (Item &it : ctx->items) {
    it.cp_off = cpoff;
    it.cp_sm = -1;
    cpoff += cp_floats(it, ctx->nx);
  }
  CK(ctx->d_cp.alloc(std::max<int64_t>(cpoff, 4)), "alloc compact iterates");
  CK(upload(ctx->d_items, ctx->items, s), "upload items");
  CK(ctx->d_N.alloc(noff), "alloc N");
  return 0;
}

// Default launch plan (the first shape that fits the shared-memory budget).
int finish_precompute(dlmpc_ctx *ctx) {
  static const int kShapes[][3] = {{128, 8, 1}, {128, 6, 1}, {128, 4, 2}, {128, 4, 1}, {128, 2, 1},
                                   {256, 2, 1}, {128, 1, 1}, {256, 1, 1}, {64, 1, 1}};
  int rc = DLMPC_ERR_ARG;
  for (const auto &sh : kShapes) {
    rc = plan_sweep(ctx, sh[0], sh[1], sh[2]);
    if (rc == 0) break;
  }
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->stream), "precompute");
  ctx->precomputed = true;
  return DLMPC_OK;
}

// Structure signature of a context's operators: nx, items, and per item the
// sizes that fix the operator layout.
uint64_t operator_signature(const dlmpc_ctx *ctx) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&h](uint64_t v) {
    h ^= v;
    h *= 1099511628211ull;
  };
  mix((uint64_t)ctx->nx);
  mix((uint64_t)ctx->nu);
  mix((uint64_t)ctx->n_sub);
  for (const Item &it : ctx->items) {
    mix((uint64_t)it.r_sub);
    mix((uint64_t)it.n_mem);
    mix((uint64_t)it.dred);
    mix((uint64_t)it.self_pos);
  }
  return h;
}

constexpr uint64_t kOperatorMagic = 0x3150504f434d4c44ull;  // "DLMCOPP1"

}  // namespace

// Blob: magic, signature, n_items, n_floats, q_floats (int64 each), k per
// item (int32), N and N^T (n_floats FP32), q (q_floats FP32).
extern "C" int64_t dlmpc_export_operators(dlmpc_ctx *ctx, void *buf, int64_t cap) {
  if (!ctx) return DLMPC_ERR_ARG;
  if (!ctx->precomputed) return ctx->fail(DLMPC_ERR_ARG, "dlmpc_precompute has not run");
  const int64_t need = 5 * 8 + (int64_t)ctx->n_sub * 4 + (ctx->n_floats + ctx->q_floats) * 4;
  if (!buf || cap < need) return need;
  auto *p = static_cast<unsigned char *>(buf);
  const int64_t head[5] = {(int64_t)kOperatorMagic, (int64_t)operator_signature(ctx), ctx->n_sub, ctx->n_floats,
                           ctx->q_floats};
  std::memcpy(p, head, sizeof head);
  p += sizeof head;
  for (const Item &it : ctx->items) {
    const int32_t k = it.k;
    std::memcpy(p, &k, 4);
    p += 4;
  }
  cudaStream_t s = ctx->stream;
  CK(cudaMemcpyAsync(p, ctx->d_N.p, ctx->n_floats * 4, cudaMemcpyDeviceToHost, s), "D2H N");
  p += ctx->n_floats * 4;
  CK(cudaMemcpyAsync(p, ctx->d_q.p, ctx->q_floats * 4, cudaMemcpyDeviceToHost, s), "D2H q");
  CK(cudaStreamSynchronize(s), "export");
  return need;
}

extern "C" int dlmpc_import_operators(dlmpc_ctx *ctx, const void *buf, int64_t size) {
  NvtxRange range("dlmpc_import_operators");
  if (!ctx || !buf || size < 40) return ctx ? ctx->fail(DLMPC_ERR_ARG, "no operator blob") : DLMPC_ERR_ARG;
  const auto *p = static_cast<const unsigned char *>(buf);
  int64_t head[5];
  std::memcpy(head, p, sizeof head);
  p += sizeof head;
  if (head[0] != (int64_t)kOperatorMagic) return ctx->fail(DLMPC_ERR_ARG, "not an operator blob");
  if (head[1] != (int64_t)operator_signature(ctx) || head[2] != ctx->n_sub)
    return ctx->fail(DLMPC_ERR_ARG, "operator blob of another problem structure");
  if (size != 40 + head[2] * 4 + (head[3] + head[4]) * 4) return ctx->fail(DLMPC_ERR_ARG, "truncated operator blob");
  int rc = upload_static(ctx);
  if (rc) return rc;
  std::vector<int32_t> nul(ctx->n_sub);
  std::memcpy(nul.data(), p, (size_t)ctx->n_sub * 4);
  p += (size_t)ctx->n_sub * 4;
  for (int g = 0; g < ctx->n_sub; ++g)
    if (nul[g] < 0 || nul[g] > ctx->kub[g]) return ctx->fail(DLMPC_ERR_ARG, "operator blob: bad null-space size");
  rc = operator_layout(ctx, nul);
  if (rc) return rc;
  if (ctx->n_floats != head[3] || ctx->q_floats != head[4])
    return ctx->fail(DLMPC_ERR_ARG, "operator blob: layout mismatch");
  cudaStream_t s = ctx->stream;
  CK(ctx->d_q.alloc(ctx->q_floats), "alloc q");
  CK(cudaMemcpyAsync(ctx->d_N.p, p, ctx->n_floats * 4, cudaMemcpyHostToDevice, s), "H2D N");
  p += ctx->n_floats * 4;
  CK(cudaMemcpyAsync(ctx->d_q.p, p, ctx->q_floats * 4, cudaMemcpyHostToDevice, s), "H2D q");
  CK(cudaStreamSynchronize(s), "import");
  return finish_precompute(ctx);
}

extern "C" int dlmpc_precompute(dlmpc_ctx *ctx) {
  NvtxRange range("dlmpc_precompute");
  if (!ctx) return DLMPC_ERR_ARG;
  const int nx = ctx->nx;
  cudaStream_t s = ctx->stream;
  if (ctx->z_stale) {
    // the plant was updated since setup: the reduced constraints again
    ctx->zrow_ptr.clear();
    ctx->zcol.clear();
    ctx->zval.clear();
    ctx->rhs.clear();
    for (Item &it : ctx->items) {
      const Instance &I = ctx->inst[it.inst];
      it.z_off = (int64_t)ctx->zrow_ptr.size();
      ctx->zrow_ptr.push_back((int64_t)ctx->zcol.size());
      ctx->rhs_off[it.sub] = (int64_t)ctx->rhs.size();
      const int m = build_reduced(I, ctx->nx, ctx->nu, it.sub - I.sub_off, ctx->zrow_ptr, ctx->zcol, ctx->zval,
                                  ctx->rhs);
      if (m < 0) return ctx->fail(DLMPC_ERR_INFEASIBLE_LOCALITY, "locality constraint infeasible");
      it.mrows = m;
    }
    ctx->z_stale = false;
  }
  int rc = upload_static(ctx);
  if (rc) return rc;
  // scratch layout for the factorisation: N with stride k_ub
  std::vector<Item> scratch = ctx->items;
  int64_t off = 0, max_D = 1, max_m = 1;
  for (int g = 0; g < ctx->n_sub; ++g) {
    Item &it = scratch[g];
    it.k = ctx->kub[g];
    it.kpad = ctx->kub[g];
    it.n_off = off;
    off += round_up((int64_t)it.dred_pad * it.kpad, 4);
    max_D = std::max<int64_t>(max_D, it.dred);
    max_m = std::max<int64_t>(max_m, it.mrows);
  }
  DevBuf<Item> d_scr;
  DevBuf<float> d_Nscr;
  DevBuf<int64_t> d_zptr, d_rhs_off;
  DevBuf<int32_t> d_zcol, d_rank, d_null;
  DevBuf<double> d_zval, d_rhs, d_ws, d_feas;
  CK(upload(d_scr, scratch, s), "upload items");
  CK(d_Nscr.alloc(off), "alloc N scratch");
  CK(ctx->d_q.alloc(ctx->q_floats), "alloc q");
  CK(upload(d_zptr, ctx->zrow_ptr, s), "upload Z");
  CK(upload(d_zcol, ctx->zcol, s), "upload Z");
  CK(upload(d_zval, ctx->zval, s), "upload Z");
  CK(upload(d_rhs, ctx->rhs, s), "upload rhs");
  CK(upload(d_rhs_off, ctx->rhs_off, s), "upload rhs");
  CK(d_rank.alloc(ctx->n_sub), "alloc");
  CK(d_null.alloc(ctx->n_sub), "alloc");
  CK(d_feas.alloc(ctx->n_sub), "alloc");
  const int64_t ws_stride = round_up(max_D * max_m + (3 + nx) * max_m + 8 * max_D + max_m / 2 + 8, 32);
  int dev = 0, sms = 1;
  CK(cudaGetDevice(&dev), "cudaGetDevice");
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "attr");
  const int64_t budget = (int64_t)8 << 30;  // factorisation workspace, freed after precompute
  // the queue: patches by decreasing work D m^2 (large ones first)
  std::vector<int32_t> order(ctx->n_sub);
  std::iota(order.begin(), order.end(), 0);
  auto work = [&](int g) { return (double)scratch[g].dred * (double)scratch[g].mrows * (double)scratch[g].mrows; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
  // four CTAs per SM (the trailing-matrix updates are memory-bound, more
  // patches in flight hide their latency), within the workspace budget
  int conc = (int)std::min<int64_t>({(int64_t)ctx->n_sub, (int64_t)sms * 4,
                                     std::max<int64_t>(1, budget / (ws_stride * 8))});
  CK(d_ws.alloc((size_t)conc * ws_stride), "alloc factor workspace");
  DevBuf<int32_t> d_order, d_next;
  CK(upload(d_order, order, s), "upload factor queue");
  CK(d_next.alloc(1), "alloc factor queue");
  CK(cudaMemsetAsync(d_next.p, 0, sizeof(int32_t), s), "memset");
  FactorParams fp{};
  fp.items = d_scr.p;
  fp.n_items = ctx->n_sub;
  fp.zrow_ptr = d_zptr.p;
  fp.zcol = d_zcol.p;
  fp.zval = d_zval.p;
  fp.rhs = d_rhs.p;
  fp.rhs_off = d_rhs_off.p;
  fp.ws = d_ws.p;
  fp.ws_stride = ws_stride;
  fp.Nmat = d_Nscr.p;
  fp.qvec = ctx->d_q.p;
  fp.feas = d_feas.p;
  fp.rank = d_rank.p;
  fp.nullity = d_null.p;
  fp.nx = nx;
  fp.use_smem = 0;
  fp.order = d_order.p;
  fp.next = d_next.p;
  // dynamic shared memory: the current Householder vector (max_D doubles)
  CK(launch_factor(fp, conc, (size_t)max_D * 8, s), "factor_kernel");
  std::vector<double> feas(ctx->n_sub);
  std::vector<int32_t> nul(ctx->n_sub);
  CK(cudaMemcpyAsync(feas.data(), d_feas.p, 8 * feas.size(), cudaMemcpyDeviceToHost, s), "D2H");
  CK(cudaMemcpyAsync(nul.data(), d_null.p, 4 * nul.size(), cudaMemcpyDeviceToHost, s), "D2H");
  CK(cudaStreamSynchronize(s), "factorisation");
  for (int g = 0; g < ctx->n_sub; ++g) {
    if (!(feas[g] <= 1e-9)) {
      char buf[160];
      snprintf(buf, sizeof buf, "subsystem %d: ||Z q - e|| = %.3e (locality infeasible)", g, feas[g]);
      return ctx->fail(DLMPC_ERR_INFEASIBLE_LOCALITY, buf);
    }
    if (nul[g] > ctx->kub[g]) return ctx->fail(DLMPC_ERR_ARG, "null-space dimension above its structural bound");
    if (nul[g] > 1000) return ctx->fail(DLMPC_ERR_ARG, "null-space dimension above 1000");
  }
  rc = operator_layout(ctx, nul);
  if (rc) return rc;
  CK(launch_repack(d_scr.p, ctx->d_items.p, ctx->n_sub, d_Nscr.p, ctx->d_N.p, s), "repack_kernel");
  CK(cudaStreamSynchronize(s), "repack");
  return finish_precompute(ctx);
}

// Plant update (Sec. IV-C, Sec. V): new rows of A and B for a few
// subsystems; only the patches that see them (their ring, d + 1 hops, holds a
// changed subsystem) are re-factorised, into scratch first, so that a failed
// update leaves the context as it was.
extern "C" int dlmpc_update_plant(dlmpc_ctx *ctx, int32_t n_changed, const int32_t *subsystems,
                                  const double *A_diag, const double *A_off, const double *B) {
  NvtxRange range("dlmpc_update_plant");
  if (!ctx) return DLMPC_ERR_ARG;
  if (!ctx->precomputed) return ctx->fail(DLMPC_ERR_ARG, "dlmpc_precompute has not run");
  if (n_changed < 1 || !subsystems || !A_diag || !B)
    return ctx->fail(DLMPC_ERR_ARG, "dlmpc_update_plant: null argument or n_changed < 1");
  const int nx = ctx->nx, nu = ctx->nu;
  cudaStream_t s = ctx->stream;
  // instance of every global subsystem
  auto inst_of = [&](int g) {
    int b = 0;
    while (b + 1 < ctx->n_inst && ctx->inst[b + 1].sub_off <= g) ++b;
    return b;
  };
  std::vector<char> seen(ctx->n_sub, 0);
  int64_t off_entries = 0;
  for (int c = 0; c < n_changed; ++c) {
    const int g = subsystems[c];
    if (g < 0 || g >= ctx->n_sub) return ctx->fail(DLMPC_ERR_ARG, "dlmpc_update_plant: subsystem out of range");
    if (seen[g]) return ctx->fail(DLMPC_ERR_ARG, "dlmpc_update_plant: subsystem listed twice");
    seen[g] = 1;
    const Instance &I = ctx->inst[inst_of(g)];
    const int i = g - I.sub_off;
    off_entries += I.adj_ptr[i + 1] - I.adj_ptr[i];
  }
  if (off_entries > 0 && !A_off) return ctx->fail(DLMPC_ERR_ARG, "dlmpc_update_plant: A_off is null");
  for (int64_t e = 0; e < (int64_t)n_changed * nx * nx; ++e)
    if (!std::isfinite(A_diag[e])) return ctx->fail(DLMPC_ERR_ARG, "dlmpc_update_plant: non-finite A_diag");
  for (int64_t e = 0; e < off_entries * nx * nx; ++e)
    if (!std::isfinite(A_off[e])) return ctx->fail(DLMPC_ERR_ARG, "dlmpc_update_plant: non-finite A_off");
  for (int64_t e = 0; e < (int64_t)n_changed * nx * nu; ++e)
    if (!std::isfinite(B[e])) return ctx->fail(DLMPC_ERR_ARG, "dlmpc_update_plant: non-finite B");
  // the new plant on copies of the affected instances (committed on success)
  std::vector<Instance> fresh = ctx->inst;
  std::vector<char> affected(ctx->n_sub, 0);
  std::vector<int> dist, touched;
  {
    const double *ao = A_off;
    for (int c = 0; c < n_changed; ++c) {
      const int g = subsystems[c];
      const int b = inst_of(g);
      Instance &I = fresh[b];
      const int i = g - I.sub_off;
      std::copy(A_diag + (int64_t)c * nx * nx, A_diag + (int64_t)(c + 1) * nx * nx,
                I.A_diag.begin() + (int64_t)i * nx * nx);
      for (int e = I.adj_ptr[i]; e < I.adj_ptr[i + 1]; ++e, ao += nx * nx)
        std::copy(ao, ao + nx * nx, I.A_off.begin() + (int64_t)e * nx * nx);
      std::copy(B + (int64_t)c * nx * nu, B + (int64_t)(c + 1) * nx * nu, I.B.begin() + (int64_t)i * nx * nu);
      // every patch whose ring holds i: its hop distance to i is at most d + 1
      dist.assign(I.n_sub, -1);
      touched.clear();
      bfs(I, i, I.d + 1, dist, touched);
      for (int j : touched) affected[I.sub_off + j] = 1;
    }
  }
  std::vector<int32_t> ids;
  for (int g = 0; g < ctx->n_sub; ++g)
    if (affected[g]) ids.push_back(g);
  const int na = (int)ids.size();
  // reduced constraints of the affected patches under the new plant, and the
  // scratch layout of their factorisation (N with stride k_ub, q compact)
  std::vector<int64_t> zptr, rhs_off(na);
  std::vector<int32_t> zcol;
  std::vector<double> zval, rhs;
  std::vector<Item> scr(na), dst(na);
  int64_t noff = 0, qoff = 0, max_D = 1, max_m = 1;
  for (int a = 0; a < na; ++a) {
    const int g = ids[a];
    const Item &it = ctx->items[g];
    const Instance &I = fresh[it.inst];
    Item sc = it;
    sc.z_off = (int64_t)zptr.size();
    zptr.push_back((int64_t)zcol.size());
    rhs_off[a] = (int64_t)rhs.size();
    const int m = build_reduced(I, nx, nu, g - I.sub_off, zptr, zcol, zval, rhs);
    if (m < 0)
      return ctx->fail(DLMPC_ERR_INFEASIBLE_LOCALITY,
                       "dlmpc_update_plant: subsystem " + std::to_string(g) + ": locality constraint infeasible");
    sc.mrows = m;
    sc.k = ctx->kub[g];
    sc.kpad = ctx->kub[g];
    sc.n_off = noff;
    noff += round_up((int64_t)sc.dred_pad * sc.kpad, 4);
    sc.q_off = qoff;
    qoff += (int64_t)nx * sc.dred_pad;
    scr[a] = sc;
    dst[a] = it;
    max_D = std::max<int64_t>(max_D, sc.dred);
    max_m = std::max<int64_t>(max_m, m);
  }
  DevBuf<Item> d_scr, d_dst;
  DevBuf<float> d_Nscr, d_qscr;
  DevBuf<int64_t> d_zptr, d_rhs_off;
  DevBuf<int32_t> d_zcol, d_rank, d_null, d_order, d_next;
  DevBuf<double> d_zval, d_rhs, d_ws, d_feas;
  CK(upload(d_scr, scr, s), "upload items");
  CK(upload(d_dst, dst, s), "upload items");
  CK(d_Nscr.alloc(std::max<int64_t>(noff, 4)), "alloc N scratch");
  CK(d_qscr.alloc(std::max<int64_t>(qoff, 4)), "alloc q scratch");
  CK(upload(d_zptr, zptr, s), "upload Z");
  CK(upload(d_zcol, zcol, s), "upload Z");
  CK(upload(d_zval, zval, s), "upload Z");
  CK(upload(d_rhs, rhs, s), "upload rhs");
  CK(upload(d_rhs_off, rhs_off, s), "upload rhs");
  CK(d_rank.alloc(na), "alloc");
  CK(d_null.alloc(na), "alloc");
  CK(d_feas.alloc(na), "alloc");
  const int64_t ws_stride = round_up(max_D * max_m + (3 + nx) * max_m + 8 * max_D + max_m / 2 + 8, 32);
  int dev = 0, sms = 1;
  CK(cudaGetDevice(&dev), "cudaGetDevice");
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "attr");
  std::vector<int32_t> order(na);
  std::iota(order.begin(), order.end(), 0);
  auto work = [&](int a) { return (double)scr[a].dred * (double)scr[a].mrows * (double)scr[a].mrows; };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
  const int conc = (int)std::min<int64_t>({(int64_t)na, (int64_t)sms * 4,
                                           std::max<int64_t>(1, ((int64_t)8 << 30) / (ws_stride * 8))});
  CK(d_ws.alloc((size_t)conc * ws_stride), "alloc factor workspace");
  CK(upload(d_order, order, s), "upload factor queue");
  CK(d_next.alloc(1), "alloc factor queue");
  CK(cudaMemsetAsync(d_next.p, 0, sizeof(int32_t), s), "memset");
  FactorParams fp{};
  fp.items = d_scr.p;
  fp.n_items = na;
  fp.zrow_ptr = d_zptr.p;
  fp.zcol = d_zcol.p;
  fp.zval = d_zval.p;
  fp.rhs = d_rhs.p;
  fp.rhs_off = d_rhs_off.p;
  fp.ws = d_ws.p;
  fp.ws_stride = ws_stride;
  fp.Nmat = d_Nscr.p;
  fp.qvec = d_qscr.p;
  fp.feas = d_feas.p;
  fp.rank = d_rank.p;
  fp.nullity = d_null.p;
  fp.nx = nx;
  fp.use_smem = 0;
  fp.order = d_order.p;
  fp.next = d_next.p;
  CK(launch_factor(fp, conc, (size_t)max_D * 8, s), "factor_kernel");
  std::vector<double> feas(na);
  std::vector<int32_t> nul(na);
  CK(cudaMemcpyAsync(feas.data(), d_feas.p, 8 * feas.size(), cudaMemcpyDeviceToHost, s), "D2H");
  CK(cudaMemcpyAsync(nul.data(), d_null.p, 4 * nul.size(), cudaMemcpyDeviceToHost, s), "D2H");
  CK(cudaStreamSynchronize(s), "factorisation");
  for (int a = 0; a < na; ++a) {
    const int g = ids[a];
    if (!(feas[a] <= 1e-9)) {
      char buf[200];
      snprintf(buf, sizeof buf, "dlmpc_update_plant: subsystem %d: ||Z q - e|| = %.3e (locality infeasible)", g,
               feas[a]);
      return ctx->fail(DLMPC_ERR_INFEASIBLE_LOCALITY, buf);
    }
    if (nul[a] != ctx->items[g].k) {
      char buf[200];
      snprintf(buf, sizeof buf,
               "dlmpc_update_plant: subsystem %d: null-space dimension %d, the operator layout has %d "
               "(set up a new context for this plant)", g, nul[a], ctx->items[g].k);
      return ctx->fail(DLMPC_ERR_ARG, buf);
    }
  }
  // commit: N and N^T repacked in place, q copied, the plant on the host and
  // on the device (dynamics, network inputs); the setup-time constraint
  // arrays are rebuilt before any later dlmpc_precompute
  CK(launch_repack(d_scr.p, d_dst.p, na, d_Nscr.p, ctx->d_N.p, s), "repack_kernel");
  for (int a = 0; a < na; ++a)
    CK(cudaMemcpyAsync(ctx->d_q.p + dst[a].q_off, d_qscr.p + scr[a].q_off, sizeof(float) * nx * dst[a].dred_pad,
                       cudaMemcpyDeviceToDevice, s),
       "copy q");
  ctx->inst.swap(fresh);
  ctx->z_stale = true;
  int64_t ad = 0, ao = 0, bm = 0;
  for (const Instance &I : ctx->inst) {
    CK(cudaMemcpyAsync(ctx->d_Adiag.p + ad, I.A_diag.data(), I.A_diag.size() * 8, cudaMemcpyHostToDevice, s), "H2D A");
    CK(cudaMemcpyAsync(ctx->d_Aoff.p + ao, I.A_off.data(), I.A_off.size() * 8, cudaMemcpyHostToDevice, s), "H2D A");
    CK(cudaMemcpyAsync(ctx->d_B.p + bm, I.B.data(), I.B.size() * 8, cudaMemcpyHostToDevice, s), "H2D B");
    ad += (int64_t)I.A_diag.size();
    ao += (int64_t)I.A_off.size();
    bm += (int64_t)I.B.size();
  }
  CK(cudaStreamSynchronize(s), "update plant");
  return na;
}

namespace {

LearnArgs learn_args(dlmpc_ctx *ctx) {
  int L = 0, slots = 1, rsub = 1;
  for (const Item &it : ctx->items) L = std::max(L, it.self_pos);
  for (const Item &it : ctx->items) {
    slots = std::max(slots, L - it.self_pos + it.n_mem);
    rsub = std::max(rsub, it.r_sub);
  }
  ctx->learn_L = L;
  ctx->learn_slots = slots;
  ctx->learn_rsub = rsub;
  LearnArgs A{ctx->d_items.p, ctx->n_sub, ctx->d_members.p, ctx->d_rev.p, ctx->nx, slots, L, rsub,
              2 * rsub * slots * ctx->nx, ctx->learn_plant, ctx->d_Adiag.p, ctx->d_Aoff.p, ctx->d_adj_ptr.p};
  return A;
}

// Learned start (Sec. V "better initial point"): network Phi~ and Lambda~ rows
// for every subsystem, then Psi0 = proj(Phi~ + Lambda~), Lambda0 = Lambda~ +
// Phi~ - Psi0 written as the starting state.
int learned_start(dlmpc_ctx *ctx, const float *x_dev) {
  if (!ctx->mlp) return ctx->fail(DLMPC_ERR_ARG, "no network attached (dlmpc_attach_mlp)");
  cudaStream_t s = ctx->stream;
  const LearnArgs A = learn_args(ctx);
  CK(launch_learn_features(A, x_dev, ctx->d_feat.p, s), "learn_features");
  // the network may run on another stream: order it between the features and
  // the scatter of its output
  const cudaStream_t ms = mlp_stream(ctx->mlp);
  if (ms != s) {
    for (auto &e : ctx->ev_learn)
      if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
    CK(cudaEventRecord(ctx->ev_learn[0], s), "event");
    CK(cudaStreamWaitEvent(ms, ctx->ev_learn[0], 0), "stream wait");
  }
  const int rc = dlmpc_mlp_forward(ctx->mlp, ctx->d_feat.p, ctx->n_sub, ctx->d_lout.p);
  if (rc) return ctx->fail(rc, std::string("network forward: ") + dlmpc_mlp_last_error(ctx->mlp));
  if (ms != s) {
    CK(cudaEventRecord(ctx->ev_learn[1], ms), "event");
    CK(cudaStreamWaitEvent(s, ctx->ev_learn[1], 0), "stream wait");
  }
  CK(launch_learn_rows(A, ctx->d_phi_l.p, ctx->d_lam.p, ctx->d_lout.p, 1, s), "learn_rows");
  CK(launch_learn_init(ctx->d_items.p, ctx->n_sub, ctx->nx, ctx->max_dred_pad, ctx->max_kpad, ctx->d_N.p, ctx->d_q.p,
                       ctx->d_phi_l.p, ctx->d_psi.p, ctx->d_lam.p, s),
     "learn_init");
  return 0;
}

Params make_params(dlmpc_ctx *ctx, const float *x_dev, float *u_dev, float *xn_dev, int warm) {
  Params P{};
  P.items = ctx->d_items.p;
  P.n_items = ctx->n_sub;
  P.grp_ptr = ctx->d_grp_ptr.p;
  P.grp_items = ctx->d_grp_items.p;
  P.cta_inst_ptr = ctx->d_cta_inst_ptr.p;
  P.cta_inst = ctx->d_cta_inst.p;
  P.members = ctx->d_members.p;
  P.rev_slot = ctx->d_rev.p;
  P.np_of = ctx->d_np.p;
  P.g_off = ctx->d_goff.p;
  P.Nmat = ctx->d_N.p;
  P.qvec = ctx->d_q.p;
  P.Psi = ctx->d_psi.p;
  P.Lam = ctx->d_lam.p;
  P.Phi = ctx->export_phi ? ctx->d_phi.p : nullptr;
  P.G0 = ctx->d_G0.p;
  P.G1 = ctx->d_G1.p;
  P.S = ctx->d_S.p;
  P.x = x_dev;
  P.u = u_dev;
  P.x_next = xn_dev;
  P.qw = ctx->d_qw.p;
  P.rw = ctx->d_rw.p;
  P.xlo = ctx->d_xlo.p;
  P.xhi = ctx->d_xhi.p;
  P.ulo = ctx->d_ulo.p;
  P.uhi = ctx->d_uhi.p;
  P.Adiag = ctx->d_Adiag.p;
  P.Aoff = ctx->d_Aoff.p;
  P.adj_ptr = ctx->d_adj_ptr.p;
  P.adj_idx = ctx->d_adj_idx.p;
  P.Bm = ctx->d_B.p;
  P.n_inst = ctx->n_inst;
  P.rho_i = ctx->d_rho.p;
  P.epsp_i = ctx->d_epsp.p;
  P.epsd_i = ctx->d_epsd.p;
  P.bar = ctx->d_bar.p;
  P.notconv = ctx->d_notconv.p;
  P.inst_iters = ctx->d_inst_iters.p;
  P.conv_prev = ctx->d_conv_prev.p;
  P.item_r = ctx->d_item_r.p;
  P.item_s = ctx->d_item_s.p;
  P.err = ctx->d_err.p;
  int max_iter = 1;
  for (const Instance &I : ctx->inst) max_iter = std::max(max_iter, I.max_iter);
  P.max_iter = ctx->max_iter_override > 0 ? ctx->max_iter_override : max_iter;
  P.fixed_iters = ctx->fixed_iters;
  P.warm = warm;
  P.nx = ctx->nx;
  P.nu = ctx->nu;
  P.timeout_ns = (unsigned long long)(ctx->timeout_ms * 1e6);
  P.ng = ctx->ng;
  P.wave = ctx->wave;
  P.max_nmem = ctx->max_nmem;
  P.max_dcol = ctx->max_dcol;
  P.max_dred_pad = ctx->max_dred_pad;
  P.max_kpad = ctx->max_kpad;
  P.grp_floats = ctx->grp_floats;
  P.cta_floats = ctx->cta_floats;
  P.max_local_inst = ctx->max_local_inst;
  P.rows_cached = ctx->rows_cached ? 1 : 0;
  P.trace = ctx->trace ? ctx->d_trace.p : nullptr;
  P.skip_arrival_cta = ctx->skip_arrival_cta;
  P.compact = ctx->compact;
  P.stale_thr = ctx->stale_thr;
  P.stale_seed = ctx->stale_seed;
  P.block_cost = (ctx->block_cost || ctx->force_block) ? 1 : 0;
  P.qblk2 = ctx->d_qblk2.p;
  P.rblk2 = ctx->d_rblk2.p;
  P.expl = ctx->coupled ? ctx->d_expl.p : nullptr;
  P.rg_base = ctx->d_rg_base.p;
  P.rg_cnt = ctx->d_rg_cnt.p;
  P.rw_base = ctx->d_rw_base.p;
  P.rw_cnt = ctx->d_rw_cnt.p;
  P.rg_desc = ctx->d_rg_desc.p;
  P.crow = ctx->d_crow.p;
  P.expl_stride = ctx->expl_stride;
  P.crow_stride = ctx->crow_stride;
  P.cpst = ctx->d_cp.p;
  return P;
}

// Sets the sweep kernel's dynamic shared-memory limit to this context's plan.
cudaError_t bind_sweep_smem(const dlmpc_ctx *ctx, bool blk) {
  const void *fn = sweep_kernel_ptr(ctx->nx, ctx->gt, blk, ctx->gt * ctx->ng);
  if (!fn) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ctx->smem);
}

// Enqueues one step: counter resets, the sweep, and (with stats) the
// statistics kernel and the copies of statistics and error words to pinned
// host memory.  `events` records the kernel-only events (not under capture).
int enqueue_step(dlmpc_ctx *ctx, const Params &P, bool with_stats, bool events, cudaStream_t s) {
  CK(cudaMemsetAsync(ctx->d_bar.p, 0, 3 * sizeof(unsigned long long), s), "memset");
  CK(cudaMemsetAsync(ctx->d_err.p, 0, 32, s), "memset");
  if (P.trace) CK(cudaMemsetAsync(ctx->d_trace.p, 0, ctx->d_trace.n * 8, s), "memset");
  if (events) CK(cudaEventRecord(ctx->ev[1], s), "event");
  CK(launch_sweep(P, ctx->gt, ctx->grid, ctx->smem, s), "sweep_kernel launch");
  if (events) CK(cudaEventRecord(ctx->ev[2], s), "event");
  if (with_stats) {
    CK(launch_stats(ctx->d_inst_item_ptr.p, ctx->n_inst, ctx->d_item_r.p, ctx->d_item_s.p, ctx->d_inst_iters.p,
                    ctx->d_err.p, ctx->fixed_iters, ctx->d_epsp.p, ctx->d_epsd.p, ctx->d_stats.p, s),
       "stats_kernel");
    CK(cudaMemcpyAsync(ctx->h_stats, ctx->d_stats.p, sizeof(dlmpc_stats) * ctx->n_inst, cudaMemcpyDeviceToHost, s),
       "D2H stats");
    CK(cudaMemcpyAsync(ctx->h_err, ctx->d_err.p, 32, cudaMemcpyDeviceToHost, s), "D2H err");
  }
  return 0;
}

// Replays (capturing on first use) the CUDA graph of one step for this set of
// pointers and options.
int graph_step(dlmpc_ctx *ctx, const Params &P, bool with_stats) {
  dlmpc_ctx::GraphKey key{P.x, P.u, P.x_next, P.warm, with_stats, ctx->plan_version, P.fixed_iters, P.max_iter,
                          P.Phi != nullptr, P.trace != nullptr, P.compact, P.block_cost, P.stale_thr,
                          P.stale_seed};
  for (auto &ge : ctx->graphs)
    if (ge.key == key) {
      CK(cudaGraphLaunch(ge.exec, ctx->stream), "cudaGraphLaunch");
      return 0;
    }
  // capture on a private stream (the caller's may be the legacy default
  // stream, which cannot be captured); the graph is launched on the caller's
  if (!ctx->capture_stream) CK(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking), "stream");
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  int rc = enqueue_step(ctx, P, with_stats, false, ctx->capture_stream);
  cudaError_t e = cudaStreamEndCapture(ctx->capture_stream, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return ctx->cuda_fail(e, "end capture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "cudaGraphInstantiate");
  if (ctx->graphs.size() >= 8) {
    cudaGraphExecDestroy(ctx->graphs.front().exec);
    ctx->graphs.erase(ctx->graphs.begin());
  }
  ctx->graphs.push_back({key, exec});
  CK(cudaGraphLaunch(exec, ctx->stream), "cudaGraphLaunch");
  return 0;
}

}  // namespace
extern "C" int dlmpc_get_timing(dlmpc_ctx *ctx, float *ms);
namespace {

int run_step(dlmpc_ctx *ctx, const float *x_dev, float *u_dev, float *xn_dev, int warm, dlmpc_stats *stats) {
  NvtxRange range(warm == DLMPC_WARM_LEARNED ? "dlmpc_step (learned start)" : "dlmpc_step");
  if (!ctx->precomputed) return ctx->fail(DLMPC_ERR_ARG, "dlmpc_precompute has not run");
  if (warm != DLMPC_WARM_COLD && warm != DLMPC_WARM_PREVIOUS && warm != DLMPC_WARM_LEARNED &&
      warm != DLMPC_WARM_CONVERGED)
    return ctx->fail(DLMPC_ERR_ARG, "unsupported warm-start mode");
  cudaStream_t s = ctx->stream;
  if (ctx->export_phi && ctx->d_phi.n != (size_t)ctx->state_floats) {
    CK(ctx->d_phi.alloc(ctx->state_floats), "alloc Phi");
    CK(cudaMemsetAsync(ctx->d_phi.p, 0, ctx->state_floats * 4, s), "memset");
  }
  if (ctx->trace) {
    const size_t n = (size_t)ctx->grid * kTraceIters * kTracePoints;
    if (ctx->d_trace.n != n) CK(ctx->d_trace.alloc(n), "alloc trace");
  }
  ctx->timed_step = false;
  if (ctx->timing) {
    for (auto &e : ctx->ev)
      if (!e) CK(cudaEventCreate(&e), "cudaEventCreate");
    CK(cudaEventRecord(ctx->ev[0], s), "event");
  }
  if (warm == DLMPC_WARM_LEARNED) {
    const int lrc = learned_start(ctx, x_dev);
    if (lrc) return lrc;
    warm = DLMPC_WARM_PREVIOUS;  // the sweep continues from the learned start
  }
  const Params P = make_params(ctx, x_dev, u_dev, xn_dev, warm);
  const bool with_stats = stats != nullptr;
  // the dynamic shared-memory limit is an attribute of the kernel function,
  // shared by every context: set this context's before its launch
  CK(bind_sweep_smem(ctx, P.block_cost != 0), "smem attr");
  ctx->kernel_events = !ctx->use_graph && ctx->timing;
  int rc = ctx->use_graph ? graph_step(ctx, P, with_stats) : enqueue_step(ctx, P, with_stats, ctx->timing != 0, s);
  if (rc) return rc;
  if (ctx->timing) {
    CK(cudaEventRecord(ctx->ev[3], s), "event");
    ctx->timed_step = true;
  }
  if (!with_stats) return DLMPC_OK;
  CK(cudaStreamSynchronize(s), "step");
  if (ctx->h_err[0] != 0) {
    char buf[200];
    snprintf(buf, sizeof buf, "device error %d (cta %d, iteration %d, aux %d)", ctx->h_err[0], ctx->h_err[1],
             ctx->h_err[2], ctx->h_err[3]);
    return ctx->fail(ctx->h_err[0], buf);
  }
  int worst = DLMPC_OK;
  for (int b = 0; b < ctx->n_inst; ++b) {
    stats[b] = ctx->h_stats[b];
    if (stats[b].status != DLMPC_OK) worst = stats[b].status;
  }
  return worst;
}

}  // namespace

extern "C" int dlmpc_step(dlmpc_ctx *ctx, const float *x_dev, float *u_dev, float *x_next_dev, int32_t warm,
                          dlmpc_stats *stats) {
  if (!ctx || !x_dev || !u_dev) return ctx ? ctx->fail(DLMPC_ERR_ARG, "null x or u") : DLMPC_ERR_ARG;
  return run_step(ctx, x_dev, u_dev, x_next_dev, warm, stats);
}

extern "C" int dlmpc_step_host(dlmpc_ctx *ctx, const float *x, float *u, float *x_next, int32_t warm,
                               dlmpc_stats *stats) {
  if (!ctx || !x || !u) return ctx ? ctx->fail(DLMPC_ERR_ARG, "null x or u") : DLMPC_ERR_ARG;
  if (!ctx->precomputed) return ctx->fail(DLMPC_ERR_ARG, "dlmpc_precompute has not run");
  cudaStream_t s = ctx->stream;
  const size_t nxb = (size_t)ctx->n_sub * ctx->nx * 4, nub = (size_t)ctx->n_sub * ctx->nu * 4;
  CK(cudaMemcpyAsync(ctx->d_x.p, x, nxb, cudaMemcpyHostToDevice, s), "H2D x");
  int rc = run_step(ctx, ctx->d_x.p, ctx->d_u.p, x_next ? ctx->d_xn.p : nullptr, warm, stats);
  if (rc < 0) return rc;
  CK(cudaMemcpyAsync(u, ctx->d_u.p, nub, cudaMemcpyDeviceToHost, s), "D2H u");
  if (x_next) CK(cudaMemcpyAsync(x_next, ctx->d_xn.p, nxb, cudaMemcpyDeviceToHost, s), "D2H x_next");
  CK(cudaStreamSynchronize(s), "step_host");
  return rc;
}

extern "C" int dlmpc_solve_batch(dlmpc_ctx *ctx, const float *const *x_dev, float *const *u_dev,
                                 float *const *x_next_dev, int32_t warm, dlmpc_stats *stats) {
  if (!ctx || !x_dev || !u_dev) return ctx ? ctx->fail(DLMPC_ERR_ARG, "null pointer table") : DLMPC_ERR_ARG;
  if (!ctx->precomputed) return ctx->fail(DLMPC_ERR_ARG, "dlmpc_precompute has not run");
  cudaStream_t s = ctx->stream;
  const int n = ctx->n_inst;
  if (ctx->d_ptr_in.n != (size_t)n) {
    CK(ctx->d_ptr_in.alloc(n), "alloc");
    CK(ctx->d_ptr_out.alloc(n), "alloc");
    CK(ctx->d_ptr_out2.alloc(n), "alloc");
  }
  std::vector<float *> xn(n, nullptr);
  if (x_next_dev)
    for (int b = 0; b < n; ++b) xn[b] = x_next_dev[b];
  CK(cudaMemcpyAsync(ctx->d_ptr_in.p, x_dev, sizeof(float *) * n, cudaMemcpyHostToDevice, s), "H2D");
  CK(cudaMemcpyAsync(ctx->d_ptr_out.p, u_dev, sizeof(float *) * n, cudaMemcpyHostToDevice, s), "H2D");
  CK(cudaMemcpyAsync(ctx->d_ptr_out2.p, xn.data(), sizeof(float *) * n, cudaMemcpyHostToDevice, s), "H2D");
  CK(launch_gather(ctx->d_ptr_in.p, ctx->d_sub_off.p, n, ctx->nx, ctx->d_x.p, s), "gather");
  int rc = run_step(ctx, ctx->d_x.p, ctx->d_u.p, x_next_dev ? ctx->d_xn.p : nullptr, warm, stats);
  if (rc < 0) return rc;
  CK(launch_scatter(ctx->d_u.p, ctx->d_sub_off.p, n, ctx->nu, ctx->d_ptr_out.p, s), "scatter");
  if (x_next_dev) CK(launch_scatter(ctx->d_xn.p, ctx->d_sub_off.p, n, ctx->nx, ctx->d_ptr_out2.p, s), "scatter");
  if (stats) CK(cudaStreamSynchronize(s), "solve_batch");
  return rc;
}

namespace {

// Best sweep launch per problem signature, shared by every context of the process.
struct TuneSig {
  int nx, nu, n_sub, n_inst, max_dcol, max_kpad, max_nmem;
  int64_t work;
  bool operator<(const TuneSig &o) const {
    return std::tie(nx, nu, n_sub, n_inst, max_dcol, max_kpad, max_nmem, work) <
           std::tie(o.nx, o.nu, o.n_sub, o.n_inst, o.max_dcol, o.max_kpad, o.max_nmem, o.work);
  }
};
std::mutex g_tune_mu;
std::map<TuneSig, dlmpc_tune_entry> g_tune_cache;

TuneSig signature(const dlmpc_ctx *ctx) {
  int64_t work = 0;
  for (const Item &it : ctx->items) work += (int64_t)it.dred * it.k;
  return {ctx->nx, ctx->nu, ctx->n_sub, ctx->n_inst, ctx->max_dcol, ctx->max_kpad, ctx->max_nmem, work};
}

}  // namespace

extern "C" int dlmpc_mlp_forward(dlmpc_mlp *mlp, const float *x_dev, int32_t n, float *y_dev);
extern "C" const char *dlmpc_mlp_last_error(dlmpc_mlp *mlp);
extern "C" int dlmpc_autotune(dlmpc_ctx *ctx, const float *x_dev, int32_t iters, dlmpc_tune_entry *entries,
                              int32_t cap) {
  NvtxRange range("dlmpc_autotune");
  if (!ctx || !x_dev) return DLMPC_ERR_ARG;
  if (!ctx->precomputed) return ctx->fail(DLMPC_ERR_ARG, "dlmpc_precompute has not run");
  const TuneSig sig = signature(ctx);
  if (iters <= 0) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto f = g_tune_cache.find(sig);
    if (f == g_tune_cache.end()) return ctx->fail(DLMPC_ERR_ARG, "no cached tuning for this problem shape");
    ctx->residency = f->second.residency;
    return plan_sweep(ctx, f->second.group_threads, f->second.groups_per_cta, f->second.wave, true);
  }
  cudaStream_t s = ctx->stream;
  // keep the caller's state and options
  DevBuf<float> psi_save, lam_save;
  const size_t bytes = (size_t)ctx->state_floats * 4;
  CK(psi_save.alloc(ctx->state_floats), "alloc");
  CK(lam_save.alloc(ctx->state_floats), "alloc");
  CK(cudaMemcpyAsync(psi_save.p, ctx->d_psi.p, bytes, cudaMemcpyDeviceToDevice, s), "save state");
  CK(cudaMemcpyAsync(lam_save.p, ctx->d_lam.p, bytes, cudaMemcpyDeviceToDevice, s), "save state");
  const int saved_fixed = ctx->fixed_iters, saved_res = ctx->residency, saved_graph = ctx->use_graph;
  const int saved_gt = ctx->gt, saved_ng = ctx->ng, saved_wave = ctx->wave;
  const int saved_timing = ctx->timing, saved_phi = ctx->export_phi, saved_trace = ctx->trace;
  ctx->fixed_iters = iters;
  ctx->use_graph = 0;
  ctx->timing = 1;
  ctx->export_phi = 0;
  ctx->trace = 0;
  std::vector<dlmpc_tune_entry> tried;
  dlmpc_tune_entry best{0, 0, 0, 0, std::numeric_limits<float>::infinity()};
  static const int kGt[] = {64, 96, 128, 256};
  static const int kNg[] = {1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 15};
  static const int kWave[] = {1, 2};
  static const int kRes[] = {2, 1};
  std::vector<std::tuple<int, int, int, int, int>> seen;
  for (int res : kRes)
    for (int gt : kGt)
      for (int ng : kNg)
        for (int wave : kWave) {
          if (gt * ng > 1024 || gt * ng < 64) continue;
          ctx->residency = res;
          if (plan_sweep(ctx, gt, ng, wave, false) != 0) continue;
          auto key = std::make_tuple(ctx->gt, ctx->ng, ctx->wave, res, ctx->grid);
          if (std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
          seen.push_back(key);
          float ms_best = std::numeric_limits<float>::infinity();
          bool ok = true;
          for (int rep = 0; rep < 2 && ok; ++rep) {
            dlmpc_stats st[1];
            std::vector<dlmpc_stats> stv(ctx->n_inst);
            if (run_step(ctx, x_dev, ctx->d_u.p, nullptr, DLMPC_WARM_COLD, stv.data()) < 0) {
              ok = false;
              break;
            }
            (void)st;
            float ms[2];
            if (dlmpc_get_timing(ctx, ms) != 0) { ok = false; break; }
            ms_best = std::min(ms_best, ms[0]);
          }
          if (!ok) continue;
          dlmpc_tune_entry e{ctx->gt, ctx->ng, ctx->wave, res, ms_best};
          tried.push_back(e);
          if (ms_best < best.ms) best = e;
        }
  ctx->fixed_iters = saved_fixed;
  ctx->use_graph = saved_graph;
  ctx->timing = saved_timing;
  ctx->export_phi = saved_phi;
  ctx->trace = saved_trace;
  CK(cudaMemcpyAsync(ctx->d_psi.p, psi_save.p, bytes, cudaMemcpyDeviceToDevice, s), "restore state");
  CK(cudaMemcpyAsync(ctx->d_lam.p, lam_save.p, bytes, cudaMemcpyDeviceToDevice, s), "restore state");
  CK(cudaStreamSynchronize(s), "autotune");
  int rc;
  if (best.group_threads == 0) {
    ctx->residency = saved_res;
    rc = plan_sweep(ctx, saved_gt, saved_ng, saved_wave, true);
    if (rc == 0) rc = ctx->fail(DLMPC_ERR_ARG, "no sweep shape could be timed");
    return rc;
  }
  ctx->residency = best.residency;
  rc = plan_sweep(ctx, best.group_threads, best.groups_per_cta, best.wave, true);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[sig] = best;
  }
  if (entries)
    for (int i = 0; i < (int)tried.size() && i < cap; ++i) entries[i] = tried[i];
  return (int)tried.size();
}

extern "C" int dlmpc_set_option(dlmpc_ctx *ctx, int32_t key, double value) {
  if (!ctx) return DLMPC_ERR_ARG;
  switch (key) {
    case DLMPC_OPT_FIXED_ITERS: ctx->fixed_iters = (int)value; return 0;
    case DLMPC_OPT_MAX_ITER: ctx->max_iter_override = (int)value; return 0;
    case DLMPC_OPT_TIMEOUT_MS:
      if (!(value > 0)) return ctx->fail(DLMPC_ERR_ARG, "timeout must be > 0");
      ctx->timeout_ms = value;
      return 0;
    case DLMPC_OPT_EXPORT_PHI: ctx->export_phi = value != 0; return 0;
    case DLMPC_OPT_TIMING: ctx->timing = value != 0; return 0;
    case DLMPC_OPT_TRACE: ctx->trace = value != 0; return 0;
    case DLMPC_OPT_GRAPH: ctx->use_graph = value != 0; return 0;
    case DLMPC_OPT_LEARN_PLANT: ctx->learn_plant = value != 0; return 0;
    case DLMPC_OPT_TEST_SKIP_ARRIVAL: ctx->skip_arrival_cta = (int)value; return 0;
    case DLMPC_OPT_COMPACT: ctx->compact = value != 0; return 0;
    case DLMPC_OPT_BLOCK_PHI: ctx->force_block = value != 0; return 0;
    case DLMPC_OPT_STALE_PROB:
      if (!(value >= 0 && value <= 1)) return ctx->fail(DLMPC_ERR_ARG, "the message-loss probability must lie in [0, 1]");
      ctx->stale_thr = (unsigned long long)(value * 9007199254740992.0);  // floor(p 2^53)
      return 0;
    case DLMPC_OPT_STALE_SEED:
      if (!(value >= 0 && value < 18446744073709551616.0) || value != std::floor(value))
        return ctx->fail(DLMPC_ERR_ARG, "the message-loss seed must be a non-negative integer");
      ctx->stale_seed = (unsigned long long)value;
      return 0;
    case DLMPC_OPT_RESIDENCY: {
      if (!(value >= 0 && value <= 2)) return ctx->fail(DLMPC_ERR_ARG, "residency must be 0, 1 or 2");
      const int old = ctx->residency;
      ctx->residency = (int)value;
      if (!ctx->precomputed) return 0;
      const int rc = plan_sweep(ctx, ctx->gt, ctx->ng, ctx->wave, true);
      if (rc == 0) return 0;
      const std::string why = ctx->err;  // keep the previous plan
      ctx->residency = old;
      plan_sweep(ctx, ctx->gt, ctx->ng, ctx->wave, true);
      return ctx->fail(rc, why);
    }
    case DLMPC_OPT_SWEEP_SHAPE: {
      // value = gt * 10000 + ng * 100 + wave
      const int v = (int)value;
      if (!ctx->precomputed) return ctx->fail(DLMPC_ERR_ARG, "set the sweep shape after dlmpc_precompute");
      const int ogt = ctx->gt, ong = ctx->ng, owave = ctx->wave;
      const int rc = plan_sweep(ctx, v / 10000, (v / 100) % 100, v % 100, true);
      if (rc == 0) return 0;
      const std::string why = ctx->err;  // keep the previous plan
      plan_sweep(ctx, ogt, ong, owave, true);
      return ctx->fail(rc, why);
    }
  }
  return ctx->fail(DLMPC_ERR_ARG, "unknown option");
}

extern "C" int dlmpc_get_info(dlmpc_ctx *ctx, dlmpc_info *info) {
  if (!ctx || !info) return DLMPC_ERR_ARG;
  info->n_inst = ctx->n_inst;
  info->n_sub_total = ctx->n_sub;
  info->nx = ctx->nx;
  info->nu = ctx->nu;
  info->n_items = ctx->n_sub;
  info->max_dcol = ctx->max_dcol;
  int maxk = 0;
  for (const Item &it : ctx->items) maxk = std::max(maxk, it.k);
  info->max_nullity = maxk;
  info->state_floats = ctx->state_floats;
  info->operator_bytes = ctx->n_floats * 4;
  info->offset_bytes = ctx->q_floats * 4;
  info->exchange_floats = ctx->g_floats;
  info->grid_ctas = ctx->grid;
  info->threads_per_cta = ctx->gt * ctx->ng;
  info->smem_bytes = (int32_t)ctx->smem;
  info->group_threads = ctx->gt;
  info->groups_per_cta = ctx->ng;
  info->wave = ctx->wave;
  info->resident_n_items = (int32_t)ctx->resident_n_items;
  info->resident_state_items = (int32_t)ctx->resident_state_items;
  // bytes one compact iteration must move per patch: N_j and N_j^T read once
  // each, the row sums of every patch row read, the patch's own row sums
  // written, lhat and R read and written, Y read and written
  int64_t bytes = 0, nbytes = 0;
  for (const Item &it : ctx->items) {
    const int64_t dcol = (int64_t)it.r_sub * it.n_mem;
    nbytes += (int64_t)it.dred * it.k * 4;           // N_j (its transpose holds the same entries)
    for (int e = 0; e < it.n_mem; ++e) bytes += (int64_t)ctx->np_of[ctx->members[it.mem_off + e]] * it.r_sub * 4;
    bytes += dcol * 4;                               // row partial sums written
    bytes += 2LL * (dcol + it.dred + it.k) * 4;      // lhat, R, Y
  }
  info->iter_bytes = bytes + 2 * nbytes;
  info->iter_bytes_min = bytes + nbytes;
  return 0;
}

extern "C" int dlmpc_learned_dims(dlmpc_ctx *ctx, int32_t *d_in, int32_t *d_out) {
  if (!ctx || !ctx->precomputed) return ctx ? ctx->fail(DLMPC_ERR_ARG, "dlmpc_precompute has not run") : DLMPC_ERR_ARG;
  const LearnArgs A = learn_args(ctx);
  if (d_in) *d_in = A.slots * (ctx->learn_plant ? ctx->nx + 2 * ctx->nx * ctx->nx : ctx->nx);
  if (d_out) *d_out = A.d_out;
  return 0;
}

extern "C" int dlmpc_learned_features(dlmpc_ctx *ctx, const float *x_dev, float *feats_dev) {
  if (!ctx || !x_dev || !feats_dev) return DLMPC_ERR_ARG;
  if (!ctx->precomputed) return ctx->fail(DLMPC_ERR_ARG, "dlmpc_precompute has not run");
  const LearnArgs A = learn_args(ctx);
  CK(launch_learn_features(A, x_dev, feats_dev, ctx->stream), "learn_features");
  return 0;
}

extern "C" int dlmpc_learned_targets(dlmpc_ctx *ctx, float *targets_dev) {
  if (!ctx || !targets_dev) return DLMPC_ERR_ARG;
  if (!ctx->d_phi.p) return ctx->fail(DLMPC_ERR_ARG, "targets need the last Phi (DLMPC_OPT_EXPORT_PHI)");
  const LearnArgs A = learn_args(ctx);
  CK(launch_learn_rows(A, ctx->d_phi.p, ctx->d_lam.p, targets_dev, 0, ctx->stream), "learn_rows");
  return 0;
}

extern "C" int dlmpc_attach_mlp(dlmpc_ctx *ctx, dlmpc_mlp *mlp) {
  if (!ctx) return DLMPC_ERR_ARG;
  if (!ctx->precomputed) return ctx->fail(DLMPC_ERR_ARG, "dlmpc_precompute has not run");
  ctx->mlp = mlp;
  if (!mlp) return 0;
  const LearnArgs A = learn_args(ctx);
  const int per = ctx->learn_plant ? ctx->nx + 2 * ctx->nx * ctx->nx : ctx->nx;
  CK(ctx->d_feat.alloc((size_t)ctx->n_sub * A.slots * per), "alloc features");
  CK(ctx->d_lout.alloc((size_t)ctx->n_sub * A.d_out), "alloc network output");
  CK(ctx->d_phi_l.alloc(ctx->state_floats), "alloc learned Phi");
  return 0;
}

// The paper's GPU mappings (Sec. III-A naive, Sec. III-C combined) for the
// ablation; variant 2 is the persistent sweep.  Runs `iters` ADMM iterations
// from a cold or previous start on x_dev and reports the host wall time.
extern "C" int dlmpc_run_variant(dlmpc_ctx *ctx, int32_t variant, const float *x_dev, int32_t iters, int32_t warm,
                                 double *ms_out) {
  if (!ctx || !x_dev || iters < 1 || variant < 0 || variant > 2 || !ms_out) return DLMPC_ERR_ARG;
  if (!ctx->precomputed) return ctx->fail(DLMPC_ERR_ARG, "dlmpc_precompute has not run");
  cudaStream_t s = ctx->stream;
  for (const Item &it : ctx->items)
    if (it.k > 256) return ctx->fail(DLMPC_ERR_ARG, "variants need null spaces of dimension <= 256");
  if (ctx->block_cost) return ctx->fail(DLMPC_ERR_ARG, "the paper variants take diagonal cost weights only");
  if (ctx->stale_thr) return ctx->fail(DLMPC_ERR_ARG, "the paper variants exchange every message");
  if (!ctx->d_phi.p || ctx->d_phi.n != (size_t)ctx->state_floats) {
    CK(ctx->d_phi.alloc(ctx->state_floats), "alloc Phi");
    CK(cudaMemsetAsync(ctx->d_phi.p, 0, ctx->state_floats * 4, s), "memset");
  }
  if (!ctx->d_psi_prev.p) CK(ctx->d_psi_prev.alloc(ctx->state_floats), "alloc");
  if (!ctx->h_exchange) CK(cudaMallocHost(&ctx->h_exchange, ctx->state_floats * 4), "alloc pinned");
  if (!ctx->d_row_sub.p) {
    std::vector<int32_t> rs, rl;
    for (int i = 0; i < ctx->n_sub; ++i)
      for (int r = 0; r < ctx->items[i].r_sub; ++r) {
        rs.push_back(i);
        rl.push_back(r);
      }
    CK(upload(ctx->d_row_sub, rs, s), "upload rows");
    CK(upload(ctx->d_row_loc, rl, s), "upload rows");
  }
  const int total_rows = (int)ctx->d_row_sub.n;
  const int64_t nst = ctx->state_floats;
  if (warm == DLMPC_WARM_COLD) {
    CK(cudaMemsetAsync(ctx->d_psi.p, 0, nst * 4, s), "memset");
    CK(cudaMemsetAsync(ctx->d_lam.p, 0, nst * 4, s), "memset");
  }
  CK(cudaStreamSynchronize(s), "variant setup");
  auto t0 = std::chrono::steady_clock::now();
  if (variant == 2) {
    const int saved_fixed = ctx->fixed_iters, saved_phi = ctx->export_phi;
    ctx->fixed_iters = iters;
    ctx->export_phi = 1;
    std::vector<dlmpc_stats> st(ctx->n_inst);
    int rc = run_step(ctx, x_dev, ctx->d_u.p, nullptr, warm == DLMPC_WARM_COLD ? DLMPC_WARM_PREVIOUS : warm, st.data());
    ctx->fixed_iters = saved_fixed;
    ctx->export_phi = saved_phi;
    if (rc < 0) return rc;
  } else {
    VariantArgs A{ctx->d_items.p, ctx->n_sub, ctx->d_members.p, ctx->d_rev.p, ctx->d_N.p, ctx->d_q.p,
                  ctx->d_phi.p, ctx->d_psi.p, ctx->d_lam.p, ctx->d_psi_prev.p, x_dev, ctx->d_S.p,
                  ctx->d_qw.p, ctx->d_rw.p, ctx->d_xlo.p, ctx->d_xhi.p, ctx->d_ulo.p, ctx->d_uhi.p,
                  ctx->d_rho.p, ctx->d_epsp.p, ctx->d_epsd.p, ctx->nx, ctx->nu, ctx->d_notconv.p};
    // information sharing through host memory, as in the paper's implementation
    auto exchange = [&](float *dev) -> int {
      CK(cudaMemcpyAsync(ctx->h_exchange, dev, nst * 4, cudaMemcpyDeviceToHost, s), "exchange D2H");
      CK(cudaMemcpyAsync(dev, ctx->h_exchange, nst * 4, cudaMemcpyHostToDevice, s), "exchange H2D");
      return 0;
    };
    CK(launch_variant_s(A, s), "variant s");
    unsigned flag = 0;
    for (int it = 0; it < iters; ++it) {
      CK(cudaMemsetAsync(ctx->d_notconv.p, 0, 4, s), "memset");
      CK(launch_variant_phi(A, ctx->d_row_sub.p, ctx->d_row_loc.p, total_rows, s), "variant phi");
      if (exchange(ctx->d_phi.p)) return DLMPC_ERR_CUDA;
      if (variant == 0) {
        CK(launch_variant_psi(A, s), "variant psi");
        if (exchange(ctx->d_psi.p)) return DLMPC_ERR_CUDA;
        CK(launch_variant_lambda(A, nst, s), "variant lambda");
        if (exchange(ctx->d_lam.p)) return DLMPC_ERR_CUDA;
        CK(launch_variant_conv(A, s), "variant conv");
      } else {
        CK(launch_variant_combined(A, s), "variant combined");
      }
      CK(cudaMemcpyAsync(&flag, ctx->d_notconv.p, 4, cudaMemcpyDeviceToHost, s), "flag");
      CK(cudaStreamSynchronize(s), "variant iteration");
    }
  }
  CK(cudaStreamSynchronize(s), "variant");
  *ms_out = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return 0;
}

extern "C" int dlmpc_get_state(dlmpc_ctx *ctx, float *phi_dev, float *psi_dev, float *lam_dev) {
  if (!ctx) return DLMPC_ERR_ARG;
  cudaStream_t s = ctx->stream;
  const size_t bytes = (size_t)ctx->state_floats * 4;
  if (phi_dev) {
    if (!ctx->d_phi.p) return ctx->fail(DLMPC_ERR_ARG, "Phi export is off (DLMPC_OPT_EXPORT_PHI)");
    CK(cudaMemcpyAsync(phi_dev, ctx->d_phi.p, bytes, cudaMemcpyDeviceToDevice, s), "copy Phi");
  }
  if (psi_dev) CK(cudaMemcpyAsync(psi_dev, ctx->d_psi.p, bytes, cudaMemcpyDeviceToDevice, s), "copy Psi");
  if (lam_dev) CK(cudaMemcpyAsync(lam_dev, ctx->d_lam.p, bytes, cudaMemcpyDeviceToDevice, s), "copy Lambda");
  return 0;
}

extern "C" int dlmpc_set_state(dlmpc_ctx *ctx, const float *psi_dev, const float *lam_dev) {
  if (!ctx || !psi_dev || !lam_dev) return DLMPC_ERR_ARG;
  if (!ctx->d_psi.p) return ctx->fail(DLMPC_ERR_ARG, "dlmpc_precompute has not run");
  cudaStream_t s = ctx->stream;
  const size_t bytes = (size_t)ctx->state_floats * 4;
  CK(cudaMemcpyAsync(ctx->d_psi.p, psi_dev, bytes, cudaMemcpyDeviceToDevice, s), "set Psi");
  CK(cudaMemcpyAsync(ctx->d_lam.p, lam_dev, bytes, cudaMemcpyDeviceToDevice, s), "set Lambda");
  // a state set by the caller is a start DLMPC_WARM_CONVERGED keeps
  const std::vector<int32_t> ones(ctx->n_inst, 1);
  CK(cudaMemcpyAsync(ctx->d_conv_prev.p, ones.data(), sizeof(int32_t) * ctx->n_inst, cudaMemcpyHostToDevice, s),
     "conv flags");
  CK(cudaStreamSynchronize(s), "set state");
  return 0;
}

extern "C" int dlmpc_get_patch(dlmpc_ctx *ctx, int32_t j, int32_t *members, int32_t cap) {
  if (!ctx || j < 0 || j >= ctx->n_sub) return DLMPC_ERR_ARG;
  const Item &it = ctx->items[j];
  if (members) {
    if (cap < it.n_mem) return ctx->fail(DLMPC_ERR_ARG, "capacity too small");
    for (int e = 0; e < it.n_mem; ++e) members[e] = ctx->members[it.mem_off + e];
  }
  return it.n_mem;
}

extern "C" int dlmpc_get_operator(dlmpc_ctx *ctx, int32_t j, double *N, int32_t n_cap, double *q, int32_t q_cap) {
  if (!ctx || j < 0 || j >= ctx->n_sub) return DLMPC_ERR_ARG;
  if (!ctx->precomputed) return ctx->fail(DLMPC_ERR_ARG, "dlmpc_precompute has not run");
  const Item &it = ctx->items[j];
  const int nx = ctx->nx, dcol = it.r_sub * it.n_mem, rsr = it.r_sub - nx;
  if ((N && n_cap < dcol * it.k) || (q && q_cap < nx * dcol)) return ctx->fail(DLMPC_ERR_ARG, "capacity too small");
  std::vector<float> hn((size_t)it.dred_pad * it.kpad), hq((size_t)nx * it.dred_pad);
  CK(cudaMemcpyAsync(hn.data(), ctx->d_N.p + it.n_off, hn.size() * 4, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
  CK(cudaMemcpyAsync(hq.data(), ctx->d_q.p + it.q_off, hq.size() * 4, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
  CK(cudaStreamSynchronize(ctx->stream), "get_operator");
  auto full = [&](int red) { const int mpos = red / rsr; return mpos * it.r_sub + nx + (red - mpos * rsr); };
  if (N) {
    std::fill(N, N + (size_t)dcol * it.k, 0.0);
    for (int red = 0; red < it.dred; ++red)
      for (int a = 0; a < it.k; ++a) N[(size_t)full(red) * it.k + a] = hn[(size_t)red * it.kpad + a];
  }
  if (q) {
    std::fill(q, q + (size_t)nx * dcol, 0.0);
    for (int c = 0; c < nx; ++c) {
      q[(size_t)c * dcol + it.self_pos * it.r_sub + c] = 1.0;
      for (int red = 0; red < it.dred; ++red) q[(size_t)c * dcol + full(red)] = hq[(size_t)c * it.dred_pad + red];
    }
  }
  return it.k;
}

extern "C" int dlmpc_get_trace(dlmpc_ctx *ctx, unsigned long long *stamps, int64_t cap) {
  if (!ctx || !stamps) return DLMPC_ERR_ARG;
  if (!ctx->d_trace.p) return ctx->fail(DLMPC_ERR_ARG, "no trace recorded (DLMPC_OPT_TRACE)");
  const int64_t n = (int64_t)ctx->d_trace.n;
  if (cap < n) return ctx->fail(DLMPC_ERR_ARG, "capacity too small");
  CK(cudaMemcpyAsync(stamps, ctx->d_trace.p, n * 8, cudaMemcpyDeviceToHost, ctx->stream), "D2H trace");
  CK(cudaStreamSynchronize(ctx->stream), "trace");
  return (int)(n / (kTraceIters * kTracePoints));
}

extern "C" int dlmpc_get_timing(dlmpc_ctx *ctx, float *ms) {
  if (!ctx || !ms) return DLMPC_ERR_ARG;
  if (!ctx->timed_step) return ctx->fail(DLMPC_ERR_ARG, "no timed step (enable DLMPC_OPT_TIMING)");
  CK(cudaEventSynchronize(ctx->ev[3]), "event sync");
  CK(cudaEventElapsedTime(&ms[1], ctx->ev[0], ctx->ev[3]), "elapsed");
  if (ctx->kernel_events) CK(cudaEventElapsedTime(&ms[0], ctx->ev[1], ctx->ev[2]), "elapsed");
  else ms[0] = ms[1];
  return 0;
}

extern "C" const char *dlmpc_last_error(dlmpc_ctx *ctx) {
  if (!ctx) return g_setup_error.c_str();
  return ctx->err.c_str();
}

extern "C" void dlmpc_destroy(dlmpc_ctx *ctx) { delete ctx; }
