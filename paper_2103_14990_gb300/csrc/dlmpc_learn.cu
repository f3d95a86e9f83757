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

#include <algorithm>

#include <cstdint>

#include "dlmpc_common.cuh"
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
// One CTA of kInitThreads per patch, all NX own columns together: T = N^T V
// (one flat pass over N for the NX vectors), psi_c = q_c + N t_c (one flat
// pass over N^T, stored after N), both read from global memory.  In: phi, lam
// hold Phi~, Lambda~; out: psi, lam hold Psi0, Lambda0.
constexpr int kInitThreads = 128;

// flat_pass (dlmpc_common.cuh) for NV right-hand sides at once: vec + c * vs
// and part + c * ps for column c.
template <int U, int NV>
__device__ __forceinline__ void flat_pass_nv(const float *M, int rows, int ld, const float *vec, int vs, float *part,
                                             int ps, int gt, int GT) {
  const int ng4 = ld >> 2;
  const int QS = GT >= ng4 ? small_div(GT, ng4) : 1;
  for (int e = gt; e < QS * ng4; e += GT) {
    const int q = small_div(e, ng4), cg = e - q * ng4;
    const float *mp = M + q * ld + 4 * cg;
    const float *vp = vec + q;
    const int step = QS * ld;
    int left = rows > q ? small_div(rows - q + QS - 1, QS) : 0;
    float4 acc[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    while (left > 0) {
      float4 m4[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        m4[u] = u < left ? *reinterpret_cast<const float4 *>(mp + u * step) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int c = 0; c < NV; ++c)
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const float vv = u < left ? vp[c * vs + u * QS] : 0.f;
          acc[c].x = fmaf(m4[u].x, vv, acc[c].x);
          acc[c].y = fmaf(m4[u].y, vv, acc[c].y);
          acc[c].z = fmaf(m4[u].z, vv, acc[c].z);
          acc[c].w = fmaf(m4[u].w, vv, acc[c].w);
        }
      mp += U * step;
      vp += U * QS;
      left -= U;
    }
#pragma unroll
    for (int c = 0; c < NV; ++c) *reinterpret_cast<float4 *>(part + c * ps + q * ld + 4 * cg) = acc[c];
  }
}

template <int NX>
__global__ void __launch_bounds__(kInitThreads) learn_init_kernel(const Item *items, int n_items, const float *Nmat,
                                                                  const float *qvec, const float *phi, float *psi,
                                                                  float *lam, int part_floats, int vpad, int tpad) {
  extern __shared__ __align__(16) float smv[];  // v [NX][vpad], t [NX][tpad], part [NX][part_floats]
  const int j = blockIdx.x;
  if (j >= n_items) return;
  const Item it = items[j];
  const int gt = threadIdx.x;
  const int dcol = it.r_sub * it.n_mem, rs_red = it.r_sub - NX;
  float *v = smv;
  float *t = smv + NX * vpad;
  float *part = t + NX * tpad;
  const float *N = Nmat + it.n_off;
  const float *NT = N + (int64_t)it.dred_pad * it.kpad;
  for (int e = gt; e < NX * it.dred_pad; e += kInitThreads) {
    const int c = small_div(e, it.dred_pad), red = e - c * it.dred_pad;
    float vv = 0.f;
    if (red < it.dred) {
      const int mpos = small_div(red, rs_red);
      const int64_t o = it.st_off + (int64_t)c * dcol + red + (mpos + 1) * NX;
      vv = phi[o] + lam[o];
    }
    v[c * vpad + red] = vv;
  }
  __syncthreads();
  flat_pass_nv<8, NX>(N, it.dred, it.kpad, v, vpad, part, part_floats, gt, kInitThreads);
  __syncthreads();
  {
    const int ncg = it.kpad >> 2;
    const int QS = kInitThreads >= ncg ? small_div(kInitThreads, ncg) : 1;
    for (int e = gt; e < NX * it.kpad; e += kInitThreads) {
      const int c = small_div(e, it.kpad), a = e - c * it.kpad;
      float s = 0.f;
      if (a < it.k)
        for (int q = 0; q < QS; ++q) s += part[c * part_floats + q * it.kpad + a];
      t[c * tpad + a] = s;
    }
  }
  __syncthreads();
  flat_pass_nv<8, NX>(NT, it.k, it.dred_pad, t, tpad, part, part_floats, gt, kInitThreads);
  __syncthreads();
  const int nrg = it.dred_pad >> 2;
  const int QS = kInitThreads >= nrg ? small_div(kInitThreads, nrg) : 1;
  for (int e = gt; e < NX * dcol; e += kInitThreads) {
    const int c = small_div(e, dcol), f = e - c * dcol;
    const int mpos = small_div(f, it.r_sub), r = f - mpos * it.r_sub;
    const int64_t o = it.st_off + (int64_t)c * dcol + f;
    const float vv = phi[o] + lam[o];
    float ps;
    if (r < NX) {
      ps = (mpos == it.self_pos && r == c) ? 1.f : 0.f;
    } else {
      const int red = mpos * rs_red + r - NX;
      float s = qvec[it.q_off + (int64_t)c * it.dred_pad + red];
      for (int q = 0; q < QS; ++q) s += part[c * part_floats + q * it.dred_pad + red];
      ps = s;
    }
    psi[o] = ps;
    lam[o] = vv - ps;
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

template <int NX>
static cudaError_t learn_init_nx(const Item *items, int n_items, int max_dred, int max_kpad, const float *Nmat,
                                 const float *qvec, const float *phi, float *psi, float *lam, cudaStream_t s) {
  // partial sums of a flat pass: at most 4 * threads, or one row when it is wider
  const int part = std::max(std::max(4 * kInitThreads, max_dred), max_kpad);
  const size_t smem = (size_t)NX * (max_dred + max_kpad + part) * 4;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(learn_init_kernel<NX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  learn_init_kernel<NX><<<n_items, kInitThreads, smem, s>>>(items, n_items, Nmat, qvec, phi, psi, lam, part, max_dred,
                                                            max_kpad);
  return cudaGetLastError();
}

cudaError_t launch_learn_init(const Item *items, int n_items, int nx, int max_dred, int max_kpad, const float *Nmat,
                              const float *qvec, const float *phi, float *psi, float *lam, cudaStream_t s) {
  switch (nx) {
    case 1: return learn_init_nx<1>(items, n_items, max_dred, max_kpad, Nmat, qvec, phi, psi, lam, s);
    case 2: return learn_init_nx<2>(items, n_items, max_dred, max_kpad, Nmat, qvec, phi, psi, lam, s);
    case 3: return learn_init_nx<3>(items, n_items, max_dred, max_kpad, Nmat, qvec, phi, psi, lam, s);
    case 4: return learn_init_nx<4>(items, n_items, max_dred, max_kpad, Nmat, qvec, phi, psi, lam, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace dlmpc
