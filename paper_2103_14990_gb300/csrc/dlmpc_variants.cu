// The paper's own GPU mappings of Alg. 2 (Sec. III), rebuilt on GB300 for the
// ablation against the persistent column-patch sweep:
//
//  naive     (Sec. III-A)  one kernel per ADMM step, one thread per row (Phi),
//                          per column (Psi), per element (Lambda), per
//                          subsystem (Conv); after every step the produced
//                          variable is shared through host memory and the
//                          Conv flag is read by the host.
//  combined  (Sec. III-C)  Phi kernel, then one kernel that does Psi, Lambda
//                          and Conv per column; one host exchange per iteration.
//
// Both work on the same column-owned Phi/Psi/Lambda arrays and operators as
// the persistent sweep and compute the same iterates.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "dlmpc_internal.h"

namespace dlmpc {

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
  unsigned *notconv;  // [1]
};

// s_i = ||x_hat_i||^2, one thread per subsystem.
__global__ void variant_s_kernel(VariantArgs A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n_items) return;
  const Item it = A.items[i];
  double s = 0.0;
  for (int mpos = 0; mpos < it.n_mem; ++mpos) {
    const int m = A.members[it.mem_off + mpos];
    for (int a = 0; a < A.nx; ++a) {
      const double v = A.x[(int64_t)m * A.nx + a];
      s += v * v;
    }
  }
  A.S[i] = (float)s;
}

// Phi-comp, one thread per row (subsystem i, local row r): the row's entries
// live in the column-owned state of every column subsystem j in Patch(i).
// Row g belongs to subsystem row_sub[g], local row row_loc[g].
__global__ void variant_phi_rows_kernel(VariantArgs A, const int32_t *row_sub, const int32_t *row_loc, int total) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int i = row_sub[g], r = row_loc[g];
  const Item it = A.items[i];
  const int nx = A.nx;
  float w = 0.f;
  for (int mpos = 0; mpos < it.n_mem; ++mpos) {
    const int j = A.members[it.mem_off + mpos];
    const Item jt = A.items[j];
    const int pos = A.rev_slot[it.mem_off + mpos];
    const int dcol = jt.r_sub * jt.n_mem;
    for (int c = 0; c < nx; ++c) {
      const int64_t e = jt.st_off + (int64_t)c * dcol + (int64_t)pos * jt.r_sub + r;
      w += (A.Psi[e] - A.Lam[e]) * A.x[(int64_t)j * nx + c];
    }
  }
  const float s = A.S[i];
  const int nxT = nx * it.T;
  float q, lo, hi;
  if (r < nxT) {
    const int a = r % nx;
    q = A.qw[i * nx + a];
    lo = r >= nx ? A.xlo[i * nx + a] : -INFINITY;
    hi = r >= nx ? A.xhi[i * nx + a] : INFINITY;
  } else {
    const int b = (r - nxT) % A.nu;
    q = A.rw[i * A.nu + b];
    lo = A.ulo[i * A.nu + b];
    hi = A.uhi[i * A.nu + b];
  }
  const float rho = A.rho_i[it.inst];
  float alpha = 0.f;
  if (s > 0.f) {
    const float z = fminf(fmaxf(rho * w / (rho + 2.f * q * s), lo), hi);
    alpha = (z - w) / s;
  }
  for (int mpos = 0; mpos < it.n_mem; ++mpos) {
    const int j = A.members[it.mem_off + mpos];
    const Item jt = A.items[j];
    const int pos = A.rev_slot[it.mem_off + mpos];
    const int dcol = jt.r_sub * jt.n_mem;
    for (int c = 0; c < nx; ++c) {
      const int64_t e = jt.st_off + (int64_t)c * dcol + (int64_t)pos * jt.r_sub + r;
      A.Phi[e] = A.Psi[e] - A.Lam[e] + alpha * A.x[(int64_t)j * nx + c];
    }
  }
}

// Psi-comp for one column (j, c), sequential in one thread: psi = q + N (N^T v).
__device__ void psi_column(const VariantArgs &A, const Item &it, int c) {
  const int nx = A.nx, dcol = it.r_sub * it.n_mem, rs_red = it.r_sub - nx;
  const float *N = A.Nmat + it.n_off;
  const int64_t base = it.st_off + (int64_t)c * dcol;
  float t[256];  // k <= 256 (checked by the host)
  for (int a = 0; a < it.k; ++a) t[a] = 0.f;
  for (int mpos = 0; mpos < it.n_mem; ++mpos)
    for (int r = nx; r < it.r_sub; ++r) {
      const int red = mpos * rs_red + r - nx;
      const float v = A.Phi[base + mpos * it.r_sub + r] + A.Lam[base + mpos * it.r_sub + r];
      for (int a = 0; a < it.k; ++a) t[a] += N[(int64_t)red * it.kpad + a] * v;
    }
  for (int mpos = 0; mpos < it.n_mem; ++mpos)
    for (int r = 0; r < it.r_sub; ++r) {
      float ps;
      if (r < nx) {
        ps = (mpos == it.self_pos && r == c) ? 1.f : 0.f;
      } else {
        const int red = mpos * rs_red + r - nx;
        ps = A.qvec[it.q_off + (int64_t)c * it.dred_pad + red];
        for (int a = 0; a < it.k; ++a) ps += N[(int64_t)red * it.kpad + a] * t[a];
      }
      A.PsiPrev[base + mpos * it.r_sub + r] = A.Psi[base + mpos * it.r_sub + r];
      A.Psi[base + mpos * it.r_sub + r] = ps;
    }
}

__global__ void variant_psi_kernel(VariantArgs A) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= A.n_items * A.nx) return;
  psi_column(A, A.items[g / A.nx], g % A.nx);
}

// Lambda-comp, one thread per element.
__global__ void variant_lambda_kernel(VariantArgs A, int64_t n) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  A.Lam[e] += A.Phi[e] - A.Psi[e];
}

// Conv for subsystem j over its own columns; counts the not-converged ones.
__device__ void conv_subsystem(const VariantArgs &A, int j) {
  const Item it = A.items[j];
  const int64_t n = (int64_t)A.nx * it.r_sub * it.n_mem;
  double rp = 0.0, rd = 0.0;
  for (int64_t e = 0; e < n; ++e) {
    const double dp = (double)A.Phi[it.st_off + e] - (double)A.Psi[it.st_off + e];
    const double dd = (double)A.Psi[it.st_off + e] - (double)A.PsiPrev[it.st_off + e];
    rp += dp * dp;
    rd += dd * dd;
  }
  const double rho = A.rho_i[it.inst];
  const double ep = A.epsp_i[it.inst], ed = A.epsd_i[it.inst];
  if (!(rp <= ep * ep && rho * rho * rd <= ed * ed)) atomicAdd(A.notconv, 1u);
}

__global__ void variant_conv_kernel(VariantArgs A) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= A.n_items) return;
  conv_subsystem(A, j);
}

// Combined kernel (Sec. III-C): per column Psi, then Lambda, then (second
// column of a subsystem done by the same thread) Conv of the subsystem.
__global__ void variant_combined_kernel(VariantArgs A) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= A.n_items) return;
  const Item it = A.items[j];
  for (int c = 0; c < A.nx; ++c) psi_column(A, it, c);
  const int64_t n = (int64_t)A.nx * it.r_sub * it.n_mem;
  for (int64_t e = 0; e < n; ++e) A.Lam[it.st_off + e] += A.Phi[it.st_off + e] - A.Psi[it.st_off + e];
  conv_subsystem(A, j);
}

cudaError_t launch_variant_s(const VariantArgs &A, cudaStream_t s) {
  variant_s_kernel<<<(A.n_items + 127) / 128, 128, 0, s>>>(A);
  return cudaGetLastError();
}
cudaError_t launch_variant_phi(const VariantArgs &A, const int32_t *row_sub, const int32_t *row_loc, int total,
                               cudaStream_t s) {
  variant_phi_rows_kernel<<<(total + 127) / 128, 128, 0, s>>>(A, row_sub, row_loc, total);
  return cudaGetLastError();
}
cudaError_t launch_variant_psi(const VariantArgs &A, cudaStream_t s) {
  variant_psi_kernel<<<(A.n_items * A.nx + 63) / 64, 64, 0, s>>>(A);
  return cudaGetLastError();
}
cudaError_t launch_variant_lambda(const VariantArgs &A, int64_t n, cudaStream_t s) {
  variant_lambda_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A, n);
  return cudaGetLastError();
}
cudaError_t launch_variant_conv(const VariantArgs &A, cudaStream_t s) {
  variant_conv_kernel<<<(A.n_items + 127) / 128, 128, 0, s>>>(A);
  return cudaGetLastError();
}
cudaError_t launch_variant_combined(const VariantArgs &A, cudaStream_t s) {
  variant_combined_kernel<<<(A.n_items + 63) / 64, 64, 0, s>>>(A);
  return cudaGetLastError();
}

}  // namespace dlmpc
