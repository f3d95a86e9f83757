// CUDA kernels of the DLMPC solver for sm_103a.
//
//  factor_kernel   one-time FP64 pivoted Householder QR of every reduced
//                  constraint block -> null-space basis N_j, min-norm offsets q_c
//                  (Alg. 1 "precompute necessities of closed-form solutions").
//  repack_kernel   copies N_j from the bound-strided scratch into the packed
//                  odd-stride layout read by the sweep.
//  admm_kernel     persistent cooperative kernel: per MPC step, the per-step
//                  precompute (s_i = ||x_hat_i||^2), every ADMM iteration of
//                  Alg. 2 (Phi-comp, Psi-comp, Lambda-comp, Conv) with one grid
//                  barrier per iteration, u(tau) and x(tau+1).
//  stats_kernel    per-instance iteration count, status and residual maxima.
#include <cuda_runtime.h>
#include <cstdint>
#include <cmath>

#include "dlmpc_internal.h"
#include "../../include/dlmpc.h"

namespace dlmpc {

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int32_t *p) {
  return *reinterpret_cast<const volatile int32_t *>(p);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Records the first error (code, CTA, iteration, aux) without overwriting it.
__device__ void set_error(int32_t *err, int code, int cta, int iter, int aux) {
  if (atomicCAS(err, 0, code) == 0) {
    err[1] = cta;
    err[2] = iter;
    err[3] = aux;
  }
}

// Grid-wide barrier for a cooperative launch.  Arrivals accumulate on one
// monotone counter; barrier number `epoch` completes when the counter reaches
// epoch * gridDim.x.  The wait is bounded by timeout_ns and also ends when any
// CTA has recorded an error; returns false in both cases.
__device__ bool grid_barrier(unsigned *bar, unsigned epoch, int32_t *err,
                             unsigned long long timeout_ns, int iter) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    const unsigned target = epoch * gridDim.x;
    const unsigned long long t0 = global_ns();
    int ok = 1;
    unsigned spins = 0;
    while (ld_acquire_u32(bar) < target) {
      if ((++spins & 63u) == 0u) {
        if (ld_volatile_i32(err) != 0) { ok = 0; break; }
        if (global_ns() - t0 > timeout_ns) {
          set_error(err, DLMPC_ERR_TIMEOUT, blockIdx.x, iter, 0);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

// --- mbarrier + bulk (1-D TMA) copy global -> shared ------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Issues one bulk copy of `bytes` (multiple of 16, both addresses 16-aligned)
// completing on `bar`.  Called by a single thread.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Bounded wait for phase `parity` of `bar`; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned long long timeout_ns) {
  const uint32_t a = smem_addr(bar);
  unsigned long long t0 = 0;
  for (unsigned spins = 0;; ++spins) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (spins == 0) t0 = global_ns();
    else if ((spins & 63u) == 0u && global_ns() - t0 > timeout_ns) return false;
  }
}

// ---------------------------------------------------------------------------
// One-time factorisation (FP64)
// ---------------------------------------------------------------------------
//
// The reduced constraint block of column patch j is Zr psi = b_c, over the
// patch variables without the slot-0 states (those equal e_c exactly).  With
// M = Zr^T (dred x mrows, column-major), a Householder QR with column pivoting
// M P = Q R reveals rank r; null(Zr) = span(Q[:, r:]) and the min-norm solution
// is Q[:, :r] y with R11^T y = (P^T b)[:r].

constexpr int kFactorThreads = 256;

__global__ void __launch_bounds__(kFactorThreads) factor_kernel(FactorParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int item_id = p.item_begin + blockIdx.x;
  if (item_id >= p.n_items) return;
  const Item it = p.items[item_id];
  const int D = it.dred;
  const int m = it.mrows;
  const int nx = p.nx;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  const int kub = it.k;  // on entry: the bound used for the scratch stride

  double *ws = p.ws + (int64_t)blockIdx.x * p.ws_stride;
  double *M = p.use_smem ? reinterpret_cast<double *>(smem_raw) : ws;  // D x m, column-major
  double *beta = ws + (int64_t)D * m;          // [m]
  double *vhead = beta + m;                    // [m]
  double *norms = vhead + m;                   // [m]
  double *y = norms + m;                       // [nx][m]
  double *vec = y + (int64_t)nx * m;           // [nwarps][D] per-warp work vectors
  int *perm = reinterpret_cast<int *>(vec + (int64_t)nwarps * D);  // [m]

  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int rank_sh;

  const int64_t *rp = p.zrow_ptr + it.z_off;
  // M = Zr^T: column rho of M is row rho of Zr.
  for (int64_t e = tid; e < (int64_t)D * m; e += blockDim.x) M[e] = 0.0;
  __syncthreads();
  for (int row = tid; row < m; row += blockDim.x) {
    for (int64_t e = rp[row]; e < rp[row + 1]; ++e) M[(int64_t)row * D + p.zcol[e]] = p.zval[e];
    perm[row] = row;
  }
  __syncthreads();
  double cmax_local = 0.0;
  for (int c = warp; c < m; c += nwarps) {
    double s = 0.0;
    for (int i = lane; i < D; i += 32) { const double v = M[(int64_t)c * D + i]; s += v * v; }
    s = warp_sum_d(s);
    if (lane == 0) norms[c] = s;
    cmax_local = fmax(cmax_local, s);
  }
  // tolerance relative to the largest initial column norm
  if (lane == 0) red_v[warp] = cmax_local;
  __syncthreads();
  if (tid == 0) {
    double mx = 0.0;
    for (int w = 0; w < nwarps; ++w) mx = fmax(mx, red_v[w]);
    red_v[31] = mx;
  }
  __syncthreads();
  const double tol2 = red_v[31] * 1e-20;  // (1e-10 relative)^2
  __syncthreads();

  const int kmax = D < m ? D : m;
  int rank = kmax;
  for (int kk = 0; kk < kmax; ++kk) {
    // pivot: largest remaining column norm
    double best = -1.0;
    int bi = kk;
    for (int c = kk + tid; c < m; c += blockDim.x) {
      const double v = norms[c];
      if (v > best) { best = v; bi = c; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double b = red_v[0];
      int i0 = red_i[0];
      for (int w = 1; w < nwarps; ++w)
        if (red_v[w] > b || (red_v[w] == b && red_i[w] < i0)) { b = red_v[w]; i0 = red_i[w]; }
      red_i[0] = i0;
      red_v[0] = b;
      rank_sh = (b <= tol2) ? kk : -1;
    }
    __syncthreads();
    if (rank_sh >= 0) { rank = rank_sh; break; }
    const int pc = red_i[0];
    if (pc != kk) {
      for (int i = tid; i < D; i += blockDim.x) {
        const double a = M[(int64_t)kk * D + i];
        M[(int64_t)kk * D + i] = M[(int64_t)pc * D + i];
        M[(int64_t)pc * D + i] = a;
      }
      if (tid == 0) {
        const int t = perm[kk]; perm[kk] = perm[pc]; perm[pc] = t;
        const double nn = norms[kk]; norms[kk] = norms[pc]; norms[pc] = nn;
      }
    }
    __syncthreads();
    // Householder vector of x = M[kk:, kk]:  H = I - beta v v^T,
    // v = x + sign(x0) ||x|| e1, beta = 1 / (||x|| (||x|| + |x0|)); H x = -sign(x0) ||x|| e1.
    if (tid == 0) {
      const double x0 = M[(int64_t)kk * D + kk];
      const double sig = sqrt(norms[kk]);
      const double sg = x0 >= 0.0 ? 1.0 : -1.0;
      vhead[kk] = x0 + sg * sig;
      beta[kk] = 1.0 / (sig * (sig + fabs(x0)));
      M[(int64_t)kk * D + kk] = -sg * sig;  // R(kk, kk)
    }
    __syncthreads();
    const double bk = beta[kk], vh = vhead[kk];
    const double *vcol = M + (int64_t)kk * D;  // v_i = vcol[i] for i > kk
    for (int c = kk + 1 + warp; c < m; c += nwarps) {
      double *col = M + (int64_t)c * D;
      double s = (lane == 0) ? vh * col[kk] : 0.0;
      for (int i = kk + 1 + lane; i < D; i += 32) s += vcol[i] * col[i];
      s = warp_sum_d(s) * bk;
      double nn = 0.0;
      if (lane == 0) col[kk] -= s * vh;
      for (int i = kk + 1 + lane; i < D; i += 32) {
        const double v = col[i] - s * vcol[i];
        col[i] = v;
        nn += v * v;
      }
      nn = warp_sum_d(nn);
      if (lane == 0) norms[c] = nn;
    }
    __syncthreads();
  }
  // rank is uniform across the block
  const int r = rank;
  const int k = D - r;

  // min-norm offsets: R11^T y = (P^T b)[:r], forward substitution, one warp per column c
  const double *rhs = p.rhs + p.rhs_off[item_id];
  for (int c = warp; c < nx; c += nwarps) {
    double *yc = y + (int64_t)c * m;
    for (int l = 0; l < r; ++l) {
      double s = 0.0;
      for (int i = lane; i < l; i += 32) s += M[(int64_t)l * D + i] * yc[i];
      s = warp_sum_d(s);
      if (lane == 0) yc[l] = (rhs[(int64_t)c * m + perm[l]] - s) / M[(int64_t)l * D + l];
      __syncwarp();
    }
  }
  __syncthreads();
  // Q applied to a vector: z <- H_0 H_1 ... H_{r-1} z  (reflectors in reverse order)
  auto apply_Q = [&](double *z) {
    for (int kk = r - 1; kk >= 0; --kk) {
      const double *vcol = M + (int64_t)kk * D;
      double s = (lane == 0) ? vhead[kk] * z[kk] : 0.0;
      for (int i = kk + 1 + lane; i < D; i += 32) s += vcol[i] * z[i];
      s = warp_sum_d(s) * beta[kk];
      if (lane == 0) z[kk] -= s * vhead[kk];
      for (int i = kk + 1 + lane; i < D; i += 32) z[i] -= s * vcol[i];
      __syncwarp();
    }
  };
  double *z = vec + (int64_t)warp * D;
  float *qout = p.qvec + it.q_off;
  for (int c = warp; c < nx; c += nwarps) {
    for (int i = lane; i < D; i += 32) z[i] = (i < r) ? y[(int64_t)c * m + i] : 0.0;
    __syncwarp();
    apply_Q(z);
    for (int i = lane; i < it.dred_pad; i += 32) qout[(int64_t)c * it.dred_pad + i] = (i < D) ? (float)z[i] : 0.f;
    // feasibility: max_row |Zr z - b_c|
    double worst = 0.0;
    for (int row = lane; row < m; row += 32) {
      double s = -rhs[(int64_t)c * m + row];
      for (int64_t e = rp[row]; e < rp[row + 1]; ++e) s += p.zval[e] * z[p.zcol[e]];
      worst = fmax(worst, fabs(s));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if (lane == 0) red_v[c] = worst;
    __syncwarp();
  }
  __syncthreads();
  if (tid == 0) {
    double f = 0.0;
    for (int c = 0; c < nx; ++c) f = fmax(f, red_v[c]);
    p.feas[item_id] = f;
    p.rank[item_id] = r;
    p.nullity[item_id] = k;
  }
  // null-space basis: columns Q e_{r+e}, written FP32 with stride kub (scratch)
  float *nout = p.Nmat + it.n_off;
  const int kw = k < kub ? k : kub;
  for (int e = warp; e < kw; e += nwarps) {
    for (int i = lane; i < D; i += 32) z[i] = (i == r + e) ? 1.0 : 0.0;
    __syncwarp();
    apply_Q(z);
    for (int i = lane; i < D; i += 32) nout[(int64_t)i * kub + e] = (float)z[i];
    __syncwarp();
  }
}

// Copies N from the scratch (stride kub, dred rows) into the packed layout
// (stride kpad, dred_pad rows, zero padding).
__global__ void repack_kernel(const Item *scratch_items, const Item *items, int n_items,
                              const float *src, float *dst) {
  const int item_id = blockIdx.x;
  if (item_id >= n_items) return;
  const Item s = scratch_items[item_id];
  const Item d = items[item_id];
  const int64_t total = (int64_t)d.dred_pad * d.kpad;
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
    const int row = (int)(e / d.kpad), col = (int)(e % d.kpad);
    float v = 0.f;
    if (row < d.dred && col < d.k) v = src[s.n_off + (int64_t)row * s.kpad + col];
    dst[d.n_off + e] = v;
  }
}

// ---------------------------------------------------------------------------
// Persistent ADMM sweep
// ---------------------------------------------------------------------------

constexpr int kSweepThreads = 256;

struct SweepSmem {
  float *nbuf;      // N rows (chunk)
  float *alpha;     // [max_dcol]  Phi-step scalars of the patch rows
  float *v;         // [NX][max_dcol]
  float *psi;       // [NX][max_dcol]
  float *t;         // [NX][max_kpad]
  float *part;      // [nsplit][NX][max_kpad]
  double *red;      // [2 * warps]
  uint64_t *mbar;
};

template <int NX>
__device__ __forceinline__ void load_chunk(const Params &P, const Item &it, SweepSmem &S, int row0, int rows,
                                           unsigned &phase, bool &ok) {
  __syncthreads();  // every reader of the previous chunk is done
  if (threadIdx.x == 0) {
    const unsigned bytes = (unsigned)rows * (unsigned)it.kpad * 4u;
    tma_load_1d(S.nbuf, P.Nmat + it.n_off + (int64_t)row0 * it.kpad, bytes, S.mbar);
  }
  bool got = mbar_wait(S.mbar, phase & 1u, P.timeout_ns);
  if (!got) set_error(P.err, DLMPC_ERR_TIMEOUT, blockIdx.x, -1, 1);
  ok = __syncthreads_and(got) != 0;
  ++phase;
}

// Processes one column patch for one ADMM iteration.  Returns false on error.
template <int NX>
__device__ bool sweep_item(const Params &P, const Item &it, SweepSmem &S, const float *Gcur, float *Gnext,
                           int slot, unsigned &phase, int iter, float rho, float eps_p, float eps_d,
                           bool init_only) {
  const int tid = threadIdx.x;
  const int nthreads = blockDim.x;
  const int r_sub = it.r_sub;
  const int dcol = r_sub * it.n_mem;
  const int rs_red = r_sub - NX;
  const int *mem = P.members + it.mem_off;
  const int *rev = P.rev_slot + it.mem_off;
  float xj[NX];
#pragma unroll
  for (int c = 0; c < NX; ++c) xj[c] = P.x[(int64_t)it.sub * NX + c];
  float *psi_g = P.Psi + it.st_off;
  float *lam_g = P.Lam + it.st_off;

  if (init_only) {
    // exchange-buffer initialisation from U = Psi - Lambda of the starting state
    for (int rho_i = tid; rho_i < dcol; rho_i += nthreads) {
      const int mpos = rho_i / r_sub, r = rho_i - mpos * r_sub;
      float g = 0.f;
#pragma unroll
      for (int c = 0; c < NX; ++c) g += (psi_g[(int64_t)c * dcol + rho_i] - lam_g[(int64_t)c * dcol + rho_i]) * xj[c];
      const int m = mem[mpos];
      Gnext[P.g_off[m] + (int64_t)rev[mpos] * r_sub + r] = g;
    }
    return true;
  }

  const bool whole = (int64_t)it.dred_pad * it.kpad <= P.smem_n_floats;
  const int chunk_rows = whole ? it.dred_pad : ((P.smem_n_floats / it.kpad) & ~3);
  bool ok = true;
  // (1) Phi-comp for every row of the patch (column-patch recomputation, Sec. III-D)
  for (int rho_i = tid; rho_i < dcol; rho_i += nthreads) {
    const int mpos = rho_i / r_sub, r = rho_i - mpos * r_sub;
    const int m = mem[mpos];
    const int np = P.np_of[m];
    const float *gp = Gcur + P.g_off[m] + r;
    float w = 0.f;
    for (int s = 0; s < np; ++s) w += __ldcg(gp + (int64_t)s * r_sub);
    const float sm = __ldcg(P.S + m);
    float qwt, lo, hi;
    if (r < NX * it.T) {
      const int a = r % NX;
      qwt = P.qw[m * NX + a];
      if (r >= NX) { lo = P.xlo[m * NX + a]; hi = P.xhi[m * NX + a]; }
      else { lo = -INFINITY; hi = INFINITY; }
    } else {
      const int b = (r - NX * it.T) % P.nu;
      qwt = P.rw[m * P.nu + b];
      lo = P.ulo[m * P.nu + b];
      hi = P.uhi[m * P.nu + b];
    }
    float alpha = 0.f, z = w;
    if (sm > 0.f) {
      const float z0 = rho * w / (rho + 2.f * qwt * sm);
      z = fminf(fmaxf(z0, lo), hi);
      alpha = (z - w) / sm;
    }
    S.alpha[rho_i] = alpha;
    if (m == it.sub && r >= NX * it.T && r < NX * it.T + P.nu) P.u[(int64_t)it.sub * P.nu + (r - NX * it.T)] = z;
  }
  __syncthreads();
  // (2) v = Phi + Lambda = Psi + alpha x_hat(col) on the own columns
  for (int rho_i = tid; rho_i < dcol; rho_i += nthreads) {
    const float a = S.alpha[rho_i];
#pragma unroll
    for (int c = 0; c < NX; ++c) S.v[c * dcol + rho_i] = psi_g[(int64_t)c * dcol + rho_i] + a * xj[c];
  }
  // (3) t = N^T v_red  (pass 1)
  // Column groups of KG <= nthreads columns (at most two, k <= 2 * nthreads);
  // nsplit threads share each column and split its rows.
  const int k = it.k, kpad = it.kpad;
  const int KG = k < nthreads ? (k > 0 ? k : 1) : nthreads;
  const int nsplit = nthreads / KG;
  const int a0 = tid % KG;
  const int split = tid / KG;
  float acc[2][NX];
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int c = 0; c < NX; ++c) acc[g][c] = 0.f;
  for (int row0 = 0; row0 < it.dred && ok; row0 += chunk_rows) {
    const int rows = min(chunk_rows, it.dred_pad - row0);
    load_chunk<NX>(P, it, S, row0, rows, phase, ok);
    if (!ok) break;
    if (split < nsplit) {
      const int rend = min(rows, it.dred - row0);
      for (int rr = split; rr < rend; rr += nsplit) {
        const int red = row0 + rr;
        const int mpos = red / rs_red;
        const int full = mpos * r_sub + NX + (red - mpos * rs_red);
        float vv[NX];
#pragma unroll
        for (int c = 0; c < NX; ++c) vv[c] = S.v[c * dcol + full];
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          const int a = g * KG + a0;
          if (a < k) {
            const float n = S.nbuf[rr * kpad + a];
#pragma unroll
            for (int c = 0; c < NX; ++c) acc[g][c] += n * vv[c];
          }
        }
      }
    }
  }
  if (!ok) return false;
  __syncthreads();
  if (split < nsplit) {
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int a = g * KG + a0;
      if (a < k) {
#pragma unroll
        for (int c = 0; c < NX; ++c) S.part[(split * NX + c) * kpad + a] = acc[g][c];
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < NX * k; e += nthreads) {
    const int c = e / k, a = e - c * k;
    float s = 0.f;
    for (int sp = 0; sp < nsplit; ++sp) s += S.part[(sp * NX + c) * kpad + a];
    S.t[c * kpad + a] = s;
  }
  __syncthreads();
  // (4) psi_red = q + N t  (pass 2); reuse the resident N when it fits
  const float *qv = P.qvec + it.q_off;
  for (int row0 = 0; row0 < it.dred && ok; row0 += chunk_rows) {
    const int rows = min(chunk_rows, it.dred_pad - row0);
    if (!whole) load_chunk<NX>(P, it, S, row0, rows, phase, ok);
    if (!ok) break;
    const int rend = min(rows, it.dred - row0);
    for (int rr = tid; rr < rend; rr += nthreads) {
      const int red = row0 + rr;
      float o[NX];
#pragma unroll
      for (int c = 0; c < NX; ++c) o[c] = qv[(int64_t)c * it.dred_pad + red];
      const float *nrow = S.nbuf + rr * kpad;
      for (int a = 0; a < k; ++a) {
        const float n = nrow[a];
#pragma unroll
        for (int c = 0; c < NX; ++c) o[c] += n * S.t[c * kpad + a];
      }
      const int mpos = red / rs_red;
      const int full = mpos * r_sub + NX + (red - mpos * rs_red);
#pragma unroll
      for (int c = 0; c < NX; ++c) S.psi[c * dcol + full] = o[c];
    }
  }
  if (!ok) return false;
  __syncthreads();
  // (5) slot-0 states are pinned to e_c; Lambda-comp; residuals; exchange partial sums
  double prim = 0.0, dual = 0.0;
  for (int rho_i = tid; rho_i < dcol; rho_i += nthreads) {
    const int mpos = rho_i / r_sub, r = rho_i - mpos * r_sub;
    float g = 0.f;
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      const float ps = (r < NX) ? ((mpos == it.self_pos && r == c) ? 1.f : 0.f) : S.psi[c * dcol + rho_i];
      const float vv = S.v[c * dcol + rho_i];
      const int64_t gi = (int64_t)c * dcol + rho_i;
      const float lam_old = lam_g[gi];
      const float psi_old = psi_g[gi];
      const float lam_new = vv - ps;
      const double dp = (double)lam_new - (double)lam_old;
      const double dd = (double)ps - (double)psi_old;
      prim += dp * dp;
      dual += dd * dd;
      lam_g[gi] = lam_new;
      psi_g[gi] = ps;
      if (P.Phi) P.Phi[it.st_off + gi] = lam_new - lam_old + ps;
      g += (2.f * ps - vv) * xj[c];
    }
    const int m = mem[mpos];
    Gnext[P.g_off[m] + (int64_t)rev[mpos] * r_sub + r] = g;
  }
  prim = warp_sum_d(prim);
  dual = warp_sum_d(dual);
  const int lane = tid & 31, warp = tid >> 5;
  if (lane == 0) { S.red[2 * warp] = prim; S.red[2 * warp + 1] = dual; }
  __syncthreads();
  if (tid == 0) {
    double pp = 0.0, dd = 0.0;
    for (int w = 0; w < (nthreads >> 5); ++w) { pp += S.red[2 * w]; dd += S.red[2 * w + 1]; }
    const float rj = (float)sqrt(pp);
    const float sj = (float)((double)rho * sqrt(dd));
    const bool conv = (rj <= eps_p) && (sj <= eps_d);
    if (!(isfinite(rj) && isfinite(sj))) set_error(P.err, DLMPC_ERR_NONFINITE, blockIdx.x, iter, it.sub);
    S.red[0] = rj;
    S.red[1] = sj;
    if (!conv) {
      atomicAdd(P.notconv + slot * (P.n_inst + 1) + it.inst, 1u);
      atomicAdd(P.notconv + slot * (P.n_inst + 1) + P.n_inst, 1u);
    }
  }
  __syncthreads();
  return true;
}

template <int NX>
__global__ void __launch_bounds__(kSweepThreads) admm_kernel(Params P, int max_dcol, int max_kpad) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SweepSmem S;
  {
    unsigned char *pp = smem_raw;
    S.nbuf = reinterpret_cast<float *>(pp); pp += (size_t)P.smem_n_floats * 4;
    S.alpha = reinterpret_cast<float *>(pp); pp += (size_t)max_dcol * 4;
    S.v = reinterpret_cast<float *>(pp); pp += (size_t)NX * max_dcol * 4;
    S.psi = reinterpret_cast<float *>(pp); pp += (size_t)NX * max_dcol * 4;
    S.t = reinterpret_cast<float *>(pp); pp += (size_t)NX * max_kpad * 4;
    // part[(split * NX + c) * kpad + a]: floor(256/k) * kpad <= 512 for k < 256,
    // kpad <= max_kpad otherwise
    S.part = reinterpret_cast<float *>(pp); pp += (size_t)NX * (2 * kSweepThreads + max_kpad) * 4;
    pp = reinterpret_cast<unsigned char *>(((uintptr_t)pp + 15) & ~(uintptr_t)15);
    S.red = reinterpret_cast<double *>(pp); pp += 2 * (kSweepThreads / 32) * 8;
    S.mbar = reinterpret_cast<uint64_t *>(pp);
  }
  if (threadIdx.x == 0) mbar_init(S.mbar, 1);
  __syncthreads();
  unsigned phase = 0;
  const int b = blockIdx.x;
  const int i0 = P.cta_ptr[b], i1 = P.cta_ptr[b + 1];
  unsigned epoch = 0;
  const int W = P.n_inst + 1;

  // prologue: s_i = ||x_hat_i||^2 (per-step precompute, Alg. 1), starting state
  for (int ii = i0; ii < i1; ++ii) {
    const Item it = P.items[P.cta_items[ii]];
    if (threadIdx.x < 32) {
      double s = 0.0;
      for (int e = threadIdx.x; e < it.n_mem * NX; e += 32) {
        const int m = P.members[it.mem_off + e / NX];
        const double xv = P.x[(int64_t)m * NX + (e % NX)];
        s += xv * xv;
      }
      s = warp_sum_d(s);
      if (threadIdx.x == 0) P.S[it.sub] = (float)s;
    }
    if (P.warm == DLMPC_WARM_COLD) {
      const int dcol = it.r_sub * it.n_mem;
      for (int e = threadIdx.x; e < NX * dcol; e += blockDim.x) {
        P.Psi[it.st_off + e] = 0.f;
        P.Lam[it.st_off + e] = 0.f;
      }
      __syncthreads();
    }
    sweep_item<NX>(P, it, S, nullptr, P.G0, 0, phase, -1, 0.f, 0.f, 0.f, true);
  }
  if (b == 0) {
    for (int e = threadIdx.x; e < 3 * W; e += blockDim.x) P.notconv[e] = 0u;
    for (int e = threadIdx.x; e < P.n_inst; e += blockDim.x) P.inst_iters[e] = 0;
  }
  bool ok = grid_barrier(P.bar, ++epoch, P.err, P.timeout_ns, -1);
  const int n_it = P.fixed_iters > 0 ? P.fixed_iters : P.max_iter;
  int iter = 0;
  for (; ok && iter < n_it; ++iter) {
    const int slot = iter % 3;
    const int prev = (iter + 2) % 3;
    if (b == 0) {
      for (int e = threadIdx.x; e < W; e += blockDim.x) P.notconv[((iter + 1) % 3) * W + e] = 0u;
    }
    const float *Gcur = (iter & 1) ? P.G1 : P.G0;
    float *Gnext = (iter & 1) ? P.G0 : P.G1;
    for (int ii = i0; ii < i1 && ok; ++ii) {
      const int idx = P.cta_items[ii];
      const Item it = P.items[idx];
      if (P.fixed_iters <= 0 && iter > 0) {
        const unsigned nc = ld_acquire_u32(P.notconv + prev * W + it.inst);
        if (nc == 0u) continue;  // this instance converged at the previous iteration
      }
      ok = sweep_item<NX>(P, it, S, Gcur, Gnext, slot, phase, iter, P.rho_i[it.inst], P.epsp_i[it.inst],
                          P.epsd_i[it.inst], false);
      if (ok && threadIdx.x == 0) {
        P.item_r[idx] = (float)S.red[0];
        P.item_s[idx] = (float)S.red[1];
      }
    }
    if (!ok) break;
    ok = grid_barrier(P.bar, ++epoch, P.err, P.timeout_ns, iter);
    if (!ok) break;
    const unsigned total = ld_acquire_u32(P.notconv + slot * W + P.n_inst);
    if (b == 0) {
      for (int e = threadIdx.x; e < P.n_inst; e += blockDim.x)
        if (P.inst_iters[e] == 0 && ld_acquire_u32(P.notconv + slot * W + e) == 0u) P.inst_iters[e] = iter + 1;
    }
    if (ld_volatile_i32(P.err) != 0) { ok = false; break; }
    if (P.fixed_iters <= 0 && total == 0u) { ++iter; break; }
  }
  if (b == 0 && threadIdx.x == 0) P.err[4] = iter;  // iterations run
  if (!ok) {
    if (threadIdx.x == 0) mbar_inval(S.mbar);
    return;
  }
  __syncthreads();
  // epilogue: x(tau+1) = A x(tau) + B u(tau) for the own subsystems (FP64)
  if (P.x_next) {
    for (int ii = i0; ii < i1; ++ii) {
      const Item it = P.items[P.cta_items[ii]];
      const int j = it.sub;
      if (threadIdx.x < NX) {
        const int a = threadIdx.x;
        double s = 0.0;
        for (int c = 0; c < NX; ++c) s += P.Adiag[((int64_t)j * NX + a) * NX + c] * (double)P.x[(int64_t)j * NX + c];
        for (int e = P.adj_ptr[j]; e < P.adj_ptr[j + 1]; ++e) {
          const int kk = P.adj_idx[e];
          for (int c = 0; c < NX; ++c) s += P.Aoff[((int64_t)e * NX + a) * NX + c] * (double)P.x[(int64_t)kk * NX + c];
        }
        for (int c = 0; c < P.nu; ++c) s += P.Bm[((int64_t)j * NX + a) * P.nu + c] * (double)P.u[(int64_t)j * P.nu + c];
        P.x_next[(int64_t)j * NX + a] = (float)s;
      }
    }
  }
  if (threadIdx.x == 0) mbar_inval(S.mbar);
}

// Per-instance statistics after a sweep.
__global__ void stats_kernel(const int32_t *inst_item_ptr, int n_inst, const float *item_r,
                             const float *item_s, const int32_t *inst_iters, const int32_t *err, int fixed,
                             const float *epsp, const float *epsd, dlmpc_stats *out) {
  const int b = blockIdx.x;
  if (b >= n_inst) return;
  float rm = 0.f, sm = 0.f;
  for (int i = inst_item_ptr[b] + threadIdx.x; i < inst_item_ptr[b + 1]; i += blockDim.x) {
    rm = fmaxf(rm, item_r[i]);
    sm = fmaxf(sm, item_s[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rm = fmaxf(rm, __shfl_xor_sync(0xffffffffu, rm, o));
    sm = fmaxf(sm, __shfl_xor_sync(0xffffffffu, sm, o));
  }
  __shared__ float sr[32], ss[32];
  if ((threadIdx.x & 31) == 0) { sr[threadIdx.x >> 5] = rm; ss[threadIdx.x >> 5] = sm; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { rm = fmaxf(rm, sr[w]); sm = fmaxf(sm, ss[w]); }
    const int run = err[4];
    const int it = inst_iters[b];
    dlmpc_stats st;
    st.r_max = rm;
    st.s_max = sm;
    if (fixed > 0) {
      // every iteration ran; converged means the last one satisfied Conv
      st.iters = run;
      st.status = (rm <= epsp[b] && sm <= epsd[b]) ? DLMPC_OK : DLMPC_MAX_ITER;
    } else {
      st.iters = it > 0 ? it : run;
      st.status = it > 0 ? DLMPC_OK : DLMPC_MAX_ITER;
    }
    out[b] = st;
  }
}

// Gathers / scatters per-instance buffers for dlmpc_solve_batch.
__global__ void gather_kernel(const float *const *src, const int32_t *off, int n_inst, int width, float *dst) {
  const int b = blockIdx.y;
  if (b >= n_inst) return;
  const int n = (off[b + 1] - off[b]) * width;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    dst[(int64_t)off[b] * width + e] = src[b][e];
}

__global__ void scatter_kernel(const float *src, const int32_t *off, int n_inst, int width, float *const *dst) {
  const int b = blockIdx.y;
  if (b >= n_inst || dst[b] == nullptr) return;
  const int n = (off[b + 1] - off[b]) * width;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    dst[b][e] = src[(int64_t)off[b] * width + e];
}

// ---------------------------------------------------------------------------
// host-callable launch wrappers
// ---------------------------------------------------------------------------

cudaError_t launch_factor(const FactorParams &p, int grid, size_t smem, cudaStream_t s) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  factor_kernel<<<grid, kFactorThreads, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_repack(const Item *scratch_items, const Item *items, int n_items, const float *src, float *dst,
                          cudaStream_t s) {
  repack_kernel<<<n_items, 256, 0, s>>>(scratch_items, items, n_items, src, dst);
  return cudaGetLastError();
}

template <int NX>
static const void *admm_fn() { return reinterpret_cast<const void *>(&admm_kernel<NX>); }

const void *admm_kernel_ptr(int nx) {
  switch (nx) {
    case 1: return admm_fn<1>();
    case 2: return admm_fn<2>();
    case 3: return admm_fn<3>();
    case 4: return admm_fn<4>();
  }
  return nullptr;
}

int sweep_threads() { return kSweepThreads; }

size_t sweep_smem_bytes(int nx, int smem_n_floats, int max_dcol, int max_kpad) {
  size_t b = (size_t)smem_n_floats * 4 + (size_t)max_dcol * 4 + 2 * (size_t)nx * max_dcol * 4 +
             (size_t)nx * max_kpad * 4 + (size_t)nx * (2 * kSweepThreads + max_kpad) * 4;
  b = (b + 15) & ~(size_t)15;
  b += 2 * (kSweepThreads / 32) * 8 + 16;
  return b;
}

cudaError_t launch_admm(int nx, const Params &P, int max_dcol, int max_kpad, int grid, size_t smem,
                        cudaStream_t s) {
  const void *fn = admm_kernel_ptr(nx);
  if (!fn) return cudaErrorInvalidValue;
  Params pc = P;
  void *args[] = {&pc, &max_dcol, &max_kpad};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kSweepThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t launch_stats(const int32_t *inst_item_ptr, int n_inst, const float *item_r, const float *item_s,
                         const int32_t *inst_iters, const int32_t *err, int fixed, const float *epsp,
                         const float *epsd, dlmpc_stats *out, cudaStream_t s) {
  stats_kernel<<<n_inst, 256, 0, s>>>(inst_item_ptr, n_inst, item_r, item_s, inst_iters, err, fixed, epsp, epsd,
                                      out);
  return cudaGetLastError();
}

cudaError_t launch_gather(const float *const *src, const int32_t *off, int n_inst, int width, float *dst,
                          cudaStream_t s) {
  gather_kernel<<<dim3(4, n_inst), 256, 0, s>>>(src, off, n_inst, width, dst);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const float *src, const int32_t *off, int n_inst, int width, float *const *dst,
                           cudaStream_t s) {
  scatter_kernel<<<dim3(4, n_inst), 256, 0, s>>>(src, off, n_inst, width, dst);
  return cudaGetLastError();
}

}  // namespace dlmpc
