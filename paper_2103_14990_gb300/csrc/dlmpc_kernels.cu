// CUDA kernels of the DLMPC solver for sm_103a.
//
//  factor_kernel   one-time FP64 pivoted Householder QR of every reduced
//                  constraint block -> null-space basis N_j, min-norm offsets q_c
//                  (Alg. 1 "precompute necessities of closed-form solutions").
//  repack_kernel   copies N_j from the bound-strided scratch into the packed
//                  odd-stride layout read by the sweep, followed by N_j^T.
//  (the persistent ADMM sweep itself is in dlmpc_sweep.cu)
//  stats_kernel    per-instance iteration count, status and residual maxima.
#include <cuda_runtime.h>
#include <cstdint>
#include <cmath>

#include "dlmpc_internal.h"
#include "dlmpc_common.cuh"

namespace dlmpc {

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

__device__ void factor_item(const FactorParams &p, int item_id) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
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
    // v_i (i > kk) staged in shared memory: every warp reads it once per column
    double *vcol = reinterpret_cast<double *>(smem_raw) + (p.use_smem ? (int64_t)D * m : 0);
    for (int i = kk + 1 + tid; i < D; i += blockDim.x) vcol[i] = M[(int64_t)kk * D + i];
    __syncthreads();
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
// Persistent: every CTA takes the next patch from a queue ordered by
// decreasing work (D m^2) until none is left, so large patches start first
// and no launch waits on its slowest patch; each CTA keeps its workspace slot.
__global__ void __launch_bounds__(kFactorThreads) factor_kernel(FactorParams p) {
  __shared__ int next_sh;
  for (;;) {
    if (threadIdx.x == 0) next_sh = atomicAdd(p.next, 1);
    __syncthreads();
    const int k = next_sh;
    __syncthreads();
    if (k >= p.n_items) break;
    factor_item(p, p.order[k]);
    __syncthreads();
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
  // N^T after N: k rows of dred_pad
  float *dt = dst + d.n_off + total;
  for (int64_t e = threadIdx.x; e < (int64_t)d.k * d.dred_pad; e += blockDim.x) {
    const int col = (int)(e / d.dred_pad), row = (int)(e % d.dred_pad);
    dt[e] = row < d.dred ? src[s.n_off + (int64_t)row * s.kpad + col] : 0.f;
  }
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
