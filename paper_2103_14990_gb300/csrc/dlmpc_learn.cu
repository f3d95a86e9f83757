// Data movement and initial projection of the learned warm start.
//
// A subsystem's network input is its patch state x_hat_i; members are placed
// by their position relative to i (slot = position - self_pos + L, with L the
// largest self position of the context), so on a chain slot o + d holds the
// subsystem o hops away and chain ends are zero padded.  The network output
// is the subsystem's Phi rows then its Lambda rows over the same slots:
// [r_sub][slots][nx] twice.  The column-owned state stores row r of i in
// column c of j at item j, column c, position of i in Patch(j), row r.
#include <cuda_runtime.h>

#include <cstdint>

#include "dlmpc_internal.h"

namespace dlmpc {

struct LearnArgs {
  const Item *items;
  int n_items;
  const int32_t *members;
  const int32_t *rev_slot;
  int nx, slots, L, max_rsub;
  int d_out;  // 2 * max_rsub * slots * nx
  int plant;  // != 0: each slot also carries A_mm and the sum of A_mk over neighbours k
  const double *Adiag, *Aoff;
  const int32_t *adj_ptr;
};

// Per slot: the member's state (nx), and with `plant` also its A_mm (nx*nx)
// and the sum of its coupling blocks A_mk (nx*nx).
__global__ void learn_features_kernel(LearnArgs A, const float *x, float *feats) {
  const int i = blockIdx.x;
  if (i >= A.n_items) return;
  const Item it = A.items[i];
  const int nx = A.nx;
  const int per = A.plant ? nx + 2 * nx * nx : nx;
  const int d_in = A.slots * per;
  for (int e = threadIdx.x; e < d_in; e += blockDim.x) feats[(int64_t)i * d_in + e] = 0.f;
  __syncthreads();
  for (int e = threadIdx.x; e < it.n_mem * per; e += blockDim.x) {
    const int mpos = e / per, f = e % per;
    const int m = A.members[it.mem_off + mpos];
    const int slot = mpos - it.self_pos + A.L;
    float v;
    if (f < nx) {
      v = x[(int64_t)m * nx + f];
    } else if (f < nx + nx * nx) {
      v = (float)A.Adiag[(int64_t)m * nx * nx + (f - nx)];
    } else {
      double s = 0.0;
      for (int q = A.adj_ptr[m]; q < A.adj_ptr[m + 1]; ++q) s += A.Aoff[(int64_t)q * nx * nx + (f - nx - nx * nx)];
      v = (float)s;
    }
    feats[(int64_t)i * d_in + slot * per + f] = v;
  }
}

// dir = 0: gather Phi/Lambda rows of every subsystem into `rows`;
// dir = 1: scatter `rows` into Phi/Lambda (column-owned).
__global__ void learn_rows_kernel(LearnArgs A, float *phi, float *lam, float *rows, int dir) {
  const int i = blockIdx.x;
  if (i >= A.n_items) return;
  const Item it = A.items[i];
  const int half = A.max_rsub * A.slots * A.nx;
  float *out = rows + (int64_t)i * A.d_out;
  if (dir == 0)
    for (int e = threadIdx.x; e < A.d_out; e += blockDim.x) out[e] = 0.f;
  __syncthreads();
  const int n = it.n_mem * it.r_sub * A.nx;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int c = e % A.nx;
    const int r = (e / A.nx) % it.r_sub;
    const int mpos = e / (A.nx * it.r_sub);
    const int j = A.members[it.mem_off + mpos];   // column subsystem (global)
    const Item jt = A.items[j];
    const int pos = A.rev_slot[it.mem_off + mpos];  // position of i in Patch(j)
    const int64_t g = jt.st_off + (int64_t)c * jt.r_sub * jt.n_mem + (int64_t)pos * jt.r_sub + r;
    const int slot = mpos - it.self_pos + A.L;
    const int o = (r * A.slots + slot) * A.nx + c;
    if (dir == 0) {
      out[o] = phi[g];
      out[half + o] = lam[g];
    } else {
      phi[g] = out[o];
      lam[g] = out[half + o];
    }
  }
}

// Psi0 = proj(v) with v = Phi~ + Lambda~ (Psi-comp), Lambda0 = v - Psi0.
// One CTA per patch; N and q from global memory.  In: phi, lam hold Phi~,
// Lambda~; out: psi, lam hold Psi0, Lambda0.
__global__ void learn_init_kernel(const Item *items, int n_items, int nx, const float *Nmat, const float *qvec,
                                  const float *phi, float *psi, float *lam) {
  extern __shared__ float smv[];  // [nx][dred] v, then [nx][kpad] t
  const int j = blockIdx.x;
  if (j >= n_items) return;
  const Item it = items[j];
  const int dcol = it.r_sub * it.n_mem, rs_red = it.r_sub - nx;
  float *v = smv;
  float *t = smv + nx * it.dred;
  const float *N = Nmat + it.n_off;
  for (int e = threadIdx.x; e < nx * dcol; e += blockDim.x) {
    const int c = e / dcol, f = e % dcol;
    const int mpos = f / it.r_sub, r = f % it.r_sub;
    if (r >= nx) v[c * it.dred + mpos * rs_red + r - nx] = phi[it.st_off + e] + lam[it.st_off + e];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nx * it.k; e += blockDim.x) {
    const int c = e / it.k, a = e % it.k;
    float s = 0.f;
    for (int red = 0; red < it.dred; ++red) s += N[(int64_t)red * it.kpad + a] * v[c * it.dred + red];
    t[c * it.kpad + a] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nx * dcol; e += blockDim.x) {
    const int c = e / dcol, f = e % dcol;
    const int mpos = f / it.r_sub, r = f % it.r_sub;
    const float vv = phi[it.st_off + e] + lam[it.st_off + e];
    float ps;
    if (r < nx) {
      ps = (mpos == it.self_pos && r == c) ? 1.f : 0.f;
    } else {
      const int red = mpos * rs_red + r - nx;
      float s = qvec[it.q_off + (int64_t)c * it.dred_pad + red];
      for (int a = 0; a < it.k; ++a) s += N[(int64_t)red * it.kpad + a] * t[c * it.kpad + a];
      ps = s;
    }
    psi[it.st_off + e] = ps;
    lam[it.st_off + e] = vv - ps;
  }
}

cudaError_t launch_learn_features(const LearnArgs &A, const float *x, float *feats, cudaStream_t s) {
  learn_features_kernel<<<A.n_items, 64, 0, s>>>(A, x, feats);
  return cudaGetLastError();
}

cudaError_t launch_learn_rows(const LearnArgs &A, float *phi, float *lam, float *rows, int dir, cudaStream_t s) {
  learn_rows_kernel<<<A.n_items, 256, 0, s>>>(A, phi, lam, rows, dir);
  return cudaGetLastError();
}

cudaError_t launch_learn_init(const Item *items, int n_items, int nx, int max_dred, int max_kpad, const float *Nmat,
                              const float *qvec, const float *phi, float *psi, float *lam, cudaStream_t s) {
  const size_t smem = (size_t)nx * (max_dred + max_kpad) * 4;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(learn_init_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  learn_init_kernel<<<n_items, 256, smem, s>>>(items, n_items, nx, Nmat, qvec, phi, psi, lam);
  return cudaGetLastError();
}

}  // namespace dlmpc
