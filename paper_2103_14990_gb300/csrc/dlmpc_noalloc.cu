// Allocation-free re-factorisation of one patch constraint block.
//
// Some callers cannot allocate device memory once their control loop runs: a
// real-time MPC thread that re-identifies one subsystem's model and must
// refresh the affected patch operators between two steps cannot afford
// cudaMalloc (it may synchronise the whole device and its latency is
// unbounded), and neither can code that only owns a fixed memory budget handed
// out at start-up.  dlmpc_factor_patch_noalloc serves them: it computes the
// same null-space basis and min-norm offsets as the one-time precomputation,
// with its workspace in a file-scope device array instead of cudaMalloc.
//
// The array lives in every GPU that loads the library, until the process
// exits.  Its device address is looked up once per device (first call on that
// device, with that device current) and cached; that first call must therefore
// come before any stream capture.  All calls share the array: calls that
// overlap on the GPU (different streams, or different host threads on one
// device) race and must be serialised by the caller.  Each call waits for its
// kernel and reports a null space wider than the caller's N buffer
// (DLMPC_ERR_CAPACITY) instead of cutting it silently.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/dlmpc.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[DLMPC_NOALLOC_MAX_DOUBLES];

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One CTA: Householder QR with column pivoting of M = Z^T (D x m, column-major)
// in `ws`, rank from a 1e-10 relative tolerance on the column norms, then
// N = Q[:, r:D] and q_c = Q[:, :r] R11^{-T} (P^T b_c)[:r].  Every scratch word
// read is written first in this launch.
__global__ void __launch_bounds__(kThreads)
factor_dense_noalloc_kernel(const double *__restrict__ Z, int m, int D, const double *__restrict__ rhs, int nrhs,
                            double *__restrict__ Nout, int k_cap, double *__restrict__ qout,
                            int32_t *__restrict__ rank_nullity, double *__restrict__ feas, double *ws) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kThreads / 32;
  double *M = ws;                               // D x m
  double *beta = M + (int64_t)D * m;            // m
  double *vhead = beta + m;                     // m
  double *norms = vhead + m;                    // m
  double *y = norms + m;                        // nrhs x m
  double *vec = y + (int64_t)nrhs * m;          // nwarps x D
  int *perm = reinterpret_cast<int *>(vec + (int64_t)nwarps * D);  // m
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int stop_at;

  // Z is row-major m x D, so row rho of Z is column rho of M.
  for (int64_t e = tid; e < (int64_t)D * m; e += kThreads) M[e] = Z[e];
  for (int c = tid; c < m; c += kThreads) perm[c] = c;
  for (int64_t e = tid; e < (int64_t)D * k_cap; e += kThreads) Nout[e] = 0.0;
  __syncthreads();
  double cmax = 0.0;
  for (int c = warp; c < m; c += nwarps) {
    double s = 0.0;
    for (int i = lane; i < D; i += 32) s += M[(int64_t)c * D + i] * M[(int64_t)c * D + i];
    s = warp_sum(s);
    if (lane == 0) norms[c] = s;
    cmax = fmax(cmax, s);
  }
  if (lane == 0) red_v[warp] = cmax;
  __syncthreads();
  if (tid == 0) {
    double mx = 0.0;
    for (int w = 0; w < nwarps; ++w) mx = fmax(mx, red_v[w]);
    red_v[31] = mx;
  }
  __syncthreads();
  const double tol2 = red_v[31] * 1e-20;
  __syncthreads();

  const int kmax = D < m ? D : m;
  int r = kmax;
  for (int kk = 0; kk < kmax; ++kk) {
    double best = -1.0;
    int bi = kk;
    for (int c = kk + tid; c < m; c += kThreads)
      if (norms[c] > best) { best = norms[c]; bi = c; }
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
      stop_at = (b <= tol2) ? kk : -1;
    }
    __syncthreads();
    if (stop_at >= 0) { r = stop_at; break; }
    const int pc = red_i[0];
    if (pc != kk) {
      for (int i = tid; i < D; i += kThreads) {
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
    if (tid == 0) {
      const double x0 = M[(int64_t)kk * D + kk];
      const double sig = sqrt(norms[kk]);
      const double sg = x0 >= 0.0 ? 1.0 : -1.0;
      vhead[kk] = x0 + sg * sig;
      beta[kk] = 1.0 / (sig * (sig + fabs(x0)));
      M[(int64_t)kk * D + kk] = -sg * sig;
    }
    __syncthreads();
    const double bk = beta[kk], vh = vhead[kk];
    const double *vcol = M + (int64_t)kk * D;
    for (int c = kk + 1 + warp; c < m; c += nwarps) {
      double *col = M + (int64_t)c * D;
      double s = (lane == 0) ? vh * col[kk] : 0.0;
      for (int i = kk + 1 + lane; i < D; i += 32) s += vcol[i] * col[i];
      s = warp_sum(s) * bk;
      if (lane == 0) col[kk] -= s * vh;
      double nn = 0.0;
      for (int i = kk + 1 + lane; i < D; i += 32) {
        const double v = col[i] - s * vcol[i];
        col[i] = v;
        nn += v * v;
      }
      nn = warp_sum(nn);
      if (lane == 0) norms[c] = nn;
    }
    __syncthreads();
  }
  const int k = D - r;
  for (int c = warp; c < nrhs; c += nwarps) {
    double *yc = y + (int64_t)c * m;
    for (int l = 0; l < r; ++l) {
      double s = 0.0;
      for (int i = lane; i < l; i += 32) s += M[(int64_t)l * D + i] * yc[i];
      s = warp_sum(s);
      if (lane == 0) yc[l] = (rhs[(int64_t)c * m + perm[l]] - s) / M[(int64_t)l * D + l];
      __syncwarp();
    }
  }
  __syncthreads();
  double *z = vec + (int64_t)warp * D;
  auto apply_Q = [&](void) {
    for (int kk = r - 1; kk >= 0; --kk) {
      const double *vcol = M + (int64_t)kk * D;
      double s = (lane == 0) ? vhead[kk] * z[kk] : 0.0;
      for (int i = kk + 1 + lane; i < D; i += 32) s += vcol[i] * z[i];
      s = warp_sum(s) * beta[kk];
      if (lane == 0) z[kk] -= s * vhead[kk];
      for (int i = kk + 1 + lane; i < D; i += 32) z[i] -= s * vcol[i];
      __syncwarp();
    }
  };
  for (int c = warp; c < nrhs; c += nwarps) {
    for (int i = lane; i < D; i += 32) z[i] = (i < r) ? y[(int64_t)c * m + i] : 0.0;
    __syncwarp();
    apply_Q();
    for (int i = lane; i < D; i += 32) qout[(int64_t)c * D + i] = z[i];
    double worst = 0.0;
    for (int row = lane; row < m; row += 32) {
      double s = -rhs[(int64_t)c * m + row];
      for (int i = 0; i < D; ++i) s += Z[(int64_t)row * D + i] * z[i];
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
    for (int c = 0; c < nrhs; ++c) f = fmax(f, red_v[c]);
    *feas = f;
    rank_nullity[0] = r;
    rank_nullity[1] = k;
  }
  const int kw = k < k_cap ? k : k_cap;
  for (int e = warp; e < kw; e += nwarps) {
    for (int i = lane; i < D; i += 32) z[i] = (i == r + e) ? 1.0 : 0.0;
    __syncwarp();
    apply_Q();
    for (int i = lane; i < D; i += 32) Nout[(int64_t)i * k_cap + e] = z[i];
    __syncwarp();
  }
}

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of the static scratch for the current device, looked up once.
cudaError_t scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int dlmpc_factor_patch_noalloc(const double *Z_dev, int32_t m, int32_t D, const double *rhs_dev,
                                          int32_t nrhs, double *N_dev, int32_t k_cap, double *q_dev,
                                          int32_t *rank_nullity_dev, double *feas_dev, void *stream) {
  if (!Z_dev || !rhs_dev || !N_dev || !q_dev || !rank_nullity_dev || !feas_dev) return DLMPC_ERR_ARG;
  if (m < 1 || D < 1 || nrhs < 1 || nrhs > 32 || k_cap < 1) return DLMPC_ERR_ARG;
  const int64_t need = (int64_t)D * m + (int64_t)(3 + nrhs) * m + 8LL * D + (m + 1) / 2 + 1;
  if (need > DLMPC_NOALLOC_MAX_DOUBLES) return DLMPC_ERR_ARG;  // block too large for the static workspace
  double *ws = nullptr;
  if (scratch_for_current_device(&ws) != cudaSuccess) return DLMPC_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  factor_dense_noalloc_kernel<<<1, kThreads, 0, st>>>(Z_dev, m, D, rhs_dev, nrhs, N_dev, k_cap, q_dev,
                                                      rank_nullity_dev, feas_dev, ws);
  if (cudaGetLastError() != cudaSuccess) return DLMPC_ERR_CUDA;
  // the nullity is known only once the factorisation has run: read it back
  // (host stack memory, no allocation) so that a basis wider than N_dev is
  // reported instead of silently cut
  int32_t rn[2] = {0, 0};
  if (cudaMemcpyAsync(rn, rank_nullity_dev, sizeof(rn), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return DLMPC_ERR_CUDA;
  return rn[1] > k_cap ? DLMPC_ERR_CAPACITY : DLMPC_OK;
}
