// Device helpers shared by the solver's CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

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
__device__ __forceinline__ void set_error(int32_t *err, int code, int cta, int iter, int aux) {
  if (atomicCAS(err, 0, code) == 0) {
    err[1] = cta;
    err[2] = iter;
    err[3] = aux;
  }
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
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
// flat matrix-vector pass (sweep and learned start)
// ---------------------------------------------------------------------------
// part[q][4g..4g+3] = sum over rows r = q, q + QS, ... of M[r][4g..4g+3] vec[r]
// for a row-major M (ld floats per row, 16-byte aligned rows): thread (q, g)
// owns one 16-byte column group and every QS-th row (QS = GT / (ld / 4)), so a
// warp reads consecutive 16-byte units; the caller adds the QS partials.

// floor(a / b) for 0 <= a < 2^16, 1 <= b < 2^12: the quotient of a + 1/2 is
// at least 1/(2b) away from an integer, far beyond the few-ulp error of the
// fast division, so the float result floors exactly (no integer division).
__device__ __forceinline__ int small_div(int a, int b) { return (int)__fdividef((float)a + 0.5f, (float)b); }

// The last `left` (< V) rows of a thread in one predicated chunk of V: the
// rows past `left` add exact zeros, so the sums equal any chunking's.
template <int V>
__device__ __forceinline__ void flat_tail(const float *mp, const float *vp, int step, int QS, int left, float4 &acc) {
  float4 m4[V];
  float vv[V];
#pragma unroll
  for (int u = 0; u < V; ++u) {
    m4[u] = u < left ? *reinterpret_cast<const float4 *>(mp + u * step) : make_float4(0.f, 0.f, 0.f, 0.f);
    vv[u] = u < left ? vp[u * QS] : 0.f;
  }
#pragma unroll
  for (int u = 0; u < V; ++u) {
    acc.x = fmaf(m4[u].x, vv[u], acc.x);
    acc.y = fmaf(m4[u].y, vv[u], acc.y);
    acc.z = fmaf(m4[u].z, vv[u], acc.z);
    acc.w = fmaf(m4[u].w, vv[u], acc.w);
  }
}

template <int U>
__device__ __forceinline__ void flat_pass(const float *M, int rows, int ld, const float *vec, float *part, int gt,
                                          int GT) {
  const int ng4 = ld >> 2;
  const int QS = GT >= ng4 ? small_div(GT, ng4) : 1;
  for (int e = gt; e < QS * ng4; e += GT) {  // one round unless ld > 4 GT
    const int q = small_div(e, ng4), cg = e - q * ng4;
    const float *mp = M + q * ld + 4 * cg;
    const float *vp = vec + q;
    const int step = QS * ld;
    int left = rows > q ? small_div(rows - q + QS - 1, QS) : 0;  // rows of this thread
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    // whole chunks of U rows without predicates (running pointers), then
    // one predicated tail chunk of U or U/2 rows
    for (; left >= U; left -= U) {
      float4 m4[U];
      float vv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        m4[u] = *reinterpret_cast<const float4 *>(mp + u * step);
        vv[u] = vp[u * QS];
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        acc.x = fmaf(m4[u].x, vv[u], acc.x);
        acc.y = fmaf(m4[u].y, vv[u], acc.y);
        acc.z = fmaf(m4[u].z, vv[u], acc.z);
        acc.w = fmaf(m4[u].w, vv[u], acc.w);
      }
      mp += U * step;
      vp += U * QS;
    }
    if (left > U / 2) flat_tail<U>(mp, vp, step, QS, left, acc);
    else if (left > 0) flat_tail<U / 2>(mp, vp, step, QS, left, acc);
    *reinterpret_cast<float4 *>(part + q * ld + 4 * cg) = acc;
  }
}

}  // namespace dlmpc
