// Persistent ADMM sweep for sm_103a: one cooperative launch per MPC step runs
// the per-step precompute, every iteration of Alg. 2 (Phi-comp, Psi-comp,
// Lambda-comp, Conv) and the dynamics of Alg. 1.
//
// Work split.  One CTA per SM; the CTA is cut into `ng` independent groups of
// GT threads that synchronise with named barriers.  Every column patch
// ("item", Sec. III-D) belongs to one group.  A group handles its items in
// waves: the Phi-step scalars of every row of the wave's patches first (all
// exchange loads of the wave in flight together), then per item the
// projection psi = q + N (N^T v) and the Lambda update.
//
// Shared memory.  Per group: the Phi-step scalars, v and psi in reduced
// order, t, per-warp partial sums, and a table of the wave's patch members
// (exchange offset, |Patch|, s_m, weights, bounds) so the Phi-step issues only
// the exchange loads.  After the groups: per-CTA counters, then the items'
// resident data placed by the host: Psi and Lambda, q and, where room remains,
// N (loaded once per launch by a 1-D bulk TMA copy).  Patches whose N is not
// resident read it from L2 with batched 16-byte loads.
//
// Iteration barrier.  Each CTA adds (1 + not_converged << 32) to one of three
// rotating 64-bit counters with a release reduction: the low half counts
// arrivals, the high half sums the not-converged patches, so the global Conv
// decision needs no extra atomic or barrier.  Every wait is bounded.
#include <cuda_runtime.h>
#include <cmath>
#include <cstdint>

#include "dlmpc_common.cuh"
#include "dlmpc_internal.h"

namespace dlmpc {

struct GroupLayout {
  int alpha, vred, psired, t, part, red, mtab, icache, mbar, total;
};

// Floats of one cached item: the Item, then rho, eps_p, eps_d, its own index.
constexpr int kItemFloats = (int)((sizeof(Item) + 3) / 4) + 4;

__host__ __device__ inline int round4(int v) { return (v + 3) & ~3; }

// Floats of one patch-member record: exchange read offset, |Patch|, 1/s (0
// when s = 0), exchange write base, then x[nx], rho/(rho + 2 q s)[nx],
// x_lo[nx], x_hi[nx], rho/(rho + 2 r s)[nu], u_lo[nu], u_hi[nu].
__host__ __device__ inline int member_record(int nx, int nu) { return 4 + 4 * nx + 3 * nu; }

// Float offsets inside one group region; the host uses the same function.
__host__ __device__ inline GroupLayout group_layout(int nx, int nu, int gt, int wave, int max_dcol, int max_dred_pad,
                                                    int max_kpad, int max_nmem) {
  GroupLayout L;
  int o = 0;
  L.alpha = o;  o += round4(wave * max_dcol);
  L.vred = o;   o += nx * max_dred_pad;
  L.psired = o; o += nx * max_dred_pad;
  L.t = o;      o += round4(nx * max_kpad);
  L.part = o;   o += (gt / 32) * nx * max_kpad;
  L.red = o;    o += round4(4 * (gt / 32));
  L.mtab = o;   o += round4(wave * max_nmem * member_record(nx, nu));
  L.icache = o; o += round4(wave * kItemFloats);
  L.mbar = o;   o += 4;
  L.total = o;
  return L;
}

// Phase stamps of group 0 of every CTA for the first iterations (diagnostics).
__device__ __forceinline__ void trace_point(const Params &P, int iter, int point) {
  if (P.trace && iter >= 0 && iter < kTraceIters && threadIdx.x == 0)
    P.trace[((size_t)blockIdx.x * kTraceIters + iter) * kTracePoints + point] = global_ns();
}

// Named barrier 1 + g (ids 1..15; the host limits a CTA to 15 groups).
__device__ __forceinline__ void group_sync(int g, int gt_threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(gt_threads) : "memory");
}

struct Group {
  float *alpha, *vred, *psired, *t, *part, *mtab, *icache;
  double *red;
  uint64_t *mbar;
  unsigned phase;  // completed bulk copies on mbar
};

// Caches the wave's items (with their instance constants) and fills the
// member records of their patches, so the iteration loop reads nothing but
// the exchange sums (and non-resident N) from global memory.
template <int NX>
__device__ __forceinline__ void fill_wave(const Params &P, const int *items, int wn, float *icache, float *mtab,
                                          int gt, int GT) {
  const int MT = member_record(NX, P.nu);
  constexpr int kItemWords = (int)((sizeof(Item) + 3) / 4);
  for (int e = gt; e < wn * kItemWords; e += GT) {
    const int wi = e / kItemWords, w = e % kItemWords;
    reinterpret_cast<uint32_t *>(icache + wi * kItemFloats)[w] =
        reinterpret_cast<const uint32_t *>(P.items + items[wi])[w];
  }
  for (int wi = gt; wi < wn; wi += GT) {
    const Item &it = P.items[items[wi]];
    float *ex = icache + wi * kItemFloats + kItemWords;
    ex[0] = P.rho_i[it.inst];
    ex[1] = P.epsp_i[it.inst];
    ex[2] = P.epsd_i[it.inst];
    reinterpret_cast<int *>(ex)[3] = items[wi];
  }
  for (int wi = 0; wi < wn; ++wi) {
    const Item &it = P.items[items[wi]];
    const float rho = P.rho_i[it.inst];
    float *tab = mtab + wi * P.max_nmem * MT;
    for (int e = gt; e < it.n_mem; e += GT) {
      const int m = P.members[it.mem_off + e];
      float *rec = tab + e * MT;
      const float sm = __ldcg(P.S + m);
      reinterpret_cast<int *>(rec)[0] = (int)P.g_off[m];
      reinterpret_cast<int *>(rec)[1] = P.np_of[m];
      rec[2] = sm > 0.f ? 1.f / sm : 0.f;
      reinterpret_cast<int *>(rec)[3] = (int)P.g_off[m] + P.rev_slot[it.mem_off + e] * it.r_sub;
#pragma unroll
      for (int a = 0; a < NX; ++a) {
        rec[4 + a] = P.x[(int64_t)m * NX + a];
        rec[4 + NX + a] = rho / (rho + 2.f * P.qw[m * NX + a] * sm);
        rec[4 + 2 * NX + a] = P.xlo[m * NX + a];
        rec[4 + 3 * NX + a] = P.xhi[m * NX + a];
      }
      for (int bb = 0; bb < P.nu; ++bb) {
        rec[4 + 4 * NX + bb] = rho / (rho + 2.f * P.rw[m * P.nu + bb] * sm);
        rec[4 + 4 * NX + P.nu + bb] = P.ulo[m * P.nu + bb];
        rec[4 + 4 * NX + 2 * P.nu + bb] = P.uhi[m * P.nu + bb];
      }
    }
  }
}

__device__ __forceinline__ const Item &cached_item(const float *icache, int wi) {
  return *reinterpret_cast<const Item *>(icache + wi * kItemFloats);
}
__device__ __forceinline__ const float *cached_extra(const float *icache, int wi) {
  return icache + wi * kItemFloats + (int)((sizeof(Item) + 3) / 4);
}

// Phi-comp for every row of one patch (Sec. II-A row problem, closed form):
// w = (Psi - Lambda)_r . x_hat from the exchange sums, z = clip(rho w / (rho +
// 2 q s), lo, hi), alpha = (z - w) / s (0 when s = 0).
template <int NX, int GT>
__device__ __forceinline__ void phi_rows(const Params &P, const Item &it, const float *tab, const float *Gcur,
                                         float *alpha_out, float rho, int gt) {
  const int r_sub = it.r_sub;
  const int dcol = r_sub * it.n_mem;
  const int nxT = NX * it.T;
  const int MT = member_record(NX, P.nu);
  const int dm = GT / r_sub, dr = GT - dm * r_sub;  // row stepping without division
  int mpos = gt / r_sub, r = gt - mpos * r_sub;
  for (int f = gt; f < dcol; f += GT) {
    const float *rec = tab + mpos * MT;
    const int goff = reinterpret_cast<const int *>(rec)[0];
    const int np = reinterpret_cast<const int *>(rec)[1];
    const float *gp = Gcur + goff + r;
    // the exchange loads are independent: issue them together, add in slot order
    float w = 0.f;
    for (int s0 = 0; s0 < np; s0 += 8) {
      float gv[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) gv[j] = (s0 + j < np) ? __ldcg(gp + (s0 + j) * r_sub) : 0.f;
#pragma unroll
      for (int j = 0; j < 8; ++j) w += gv[j];
    }
    const float inv_s = rec[2];
    float den, lo, hi;
    if (r < nxT) {
      const int a = r % NX;
      den = rec[4 + NX + a];
      if (r >= NX) {
        lo = rec[4 + 2 * NX + a];
        hi = rec[4 + 3 * NX + a];
      } else {
        lo = -INFINITY;
        hi = INFINITY;
      }
    } else {
      const int bb = (r - nxT) % P.nu;
      den = rec[4 + 4 * NX + bb];
      lo = rec[4 + 4 * NX + P.nu + bb];
      hi = rec[4 + 4 * NX + 2 * P.nu + bb];
    }
    // z* = rho w / (rho + 2 q s), clipped; alpha = (z - w) / s; s = 0 gives phi = v
    float a = 0.f, z = w;
    if (inv_s > 0.f) {
      z = fminf(fmaxf(w * den, lo), hi);
      a = (z - w) * inv_s;
    }
    alpha_out[f] = a;
    if (mpos == it.self_pos && r >= nxT && r < nxT + P.nu) P.u[(int64_t)it.sub * P.nu + (r - nxT)] = z;
    mpos += dm;
    r += dr;
    if (r >= r_sub) { r -= r_sub; ++mpos; }
  }
}

// Psi-comp, Lambda-comp and the residuals of one patch.
template <int NX, int GT>
__device__ void project_item(const Params &P, int idx, const Item &it, const float *tab, const float *extra, Group &G,
                             const float *alpha, float *arena, float *Gnext, int g, int gt, unsigned *lnc, int iter,
                             bool tr) {
  const float rho = extra[0];
  const int MT = member_record(NX, P.nu);
  const int r_sub = it.r_sub;
  const int dcol = r_sub * it.n_mem;
  const int rs_red = r_sub - NX;
  const int dred = it.dred;
  const int k = it.k, kpad = it.kpad;
  const int ldr = P.max_dred_pad;
  constexpr int kWarps = GT / 32;
  float *psi_p = it.st_sm >= 0 ? arena + it.st_sm : P.Psi + it.st_off;
  float *lam_p = it.st_sm >= 0 ? arena + it.st_sm + NX * dcol : P.Lam + it.st_off;
  const float *q_p = it.q_sm >= 0 ? arena + it.q_sm : P.qvec + it.q_off;
  float xj[NX];
#pragma unroll
  for (int c = 0; c < NX; ++c) xj[c] = tab[it.self_pos * MT + 4 + c];

  // v = Phi + Lambda = Psi + alpha x_hat(col), kept for the reduced rows
  const int dm = GT / r_sub, dr = GT - dm * r_sub;  // row stepping without division
  const int mpos0 = gt / r_sub, r0 = gt - mpos0 * r_sub;
  for (int f = gt, mpos = mpos0, r = r0; f < dcol; f += GT, mpos += dm, r += dr) {
    if (r >= r_sub) { r -= r_sub; ++mpos; }
    if (r >= NX) {
      const int red = mpos * rs_red + r - NX;
      const float a = alpha[f];
#pragma unroll
      for (int c = 0; c < NX; ++c) G.vred[c * ldr + red] = psi_p[c * dcol + f] + a * xj[c];
    }
  }
  // N: resident in the arena, otherwise read from global memory (L2); the
  // generic 16-byte loads below serve both.
  const float *Nb = it.n_sm >= 0 ? arena + it.n_sm : P.Nmat + it.n_off;
  group_sync(g, GT);
  if (tr) trace_point(P, iter, 6);

  // pass 1: t = N^T v.  Warp w takes row pairs (2i, 2i+1), i = w mod kWarps;
  // the half warp picks the row, the lane a group of 4 columns (blocks of 16
  // groups).  Rows are loaded 4 at a time before use.  Half warps are combined
  // by a shuffle, warps through shared memory.
  const int ncg = kpad >> 2;
  {
    const int lane = gt & 31, w = gt >> 5, hw = lane >> 4, l16 = lane & 15;
    constexpr int kStep = 2 * kWarps;
    for (int cb = 0; cb < ncg; cb += 16) {
      const int cg = cb + l16;
      float acc[4][NX];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int c = 0; c < NX; ++c) acc[j][c] = 0.f;
      if (cg < ncg) {
        const float *nb = Nb + 4 * cg;
        for (int r0 = 2 * w + hw; r0 < dred; r0 += 4 * kStep) {
          float4 n4[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int red = r0 + u * kStep;
            n4[u] = red < dred ? *reinterpret_cast<const float4 *>(nb + red * kpad) : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int red = r0 + u * kStep;
            if (red < dred) {
#pragma unroll
              for (int c = 0; c < NX; ++c) {
                const float vv = G.vred[c * ldr + red];
                acc[0][c] = fmaf(n4[u].x, vv, acc[0][c]);
                acc[1][c] = fmaf(n4[u].y, vv, acc[1][c]);
                acc[2][c] = fmaf(n4[u].z, vv, acc[2][c]);
                acc[3][c] = fmaf(n4[u].w, vv, acc[3][c]);
              }
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int c = 0; c < NX; ++c) acc[j][c] += __shfl_xor_sync(0xffffffffu, acc[j][c], 16);
      if (hw == 0 && cg < ncg) {
#pragma unroll
        for (int c = 0; c < NX; ++c)
          *reinterpret_cast<float4 *>(G.part + (w * NX + c) * kpad + 4 * cg) =
              make_float4(acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
      }
    }
  }
  group_sync(g, GT);
  for (int e = gt; e < NX * kpad; e += GT) {
    const int c = e / kpad, a = e - c * kpad;
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += G.part[(w * NX + c) * kpad + a];
    G.t[c * kpad + a] = (a < k) ? s : 0.f;  // padded columns of N are zero; keep t finite there
  }
  group_sync(g, GT);
  if (tr) trace_point(P, iter, 7);

  // pass 2: psi_red = q + N t.  16 consecutive rows per half warp (conflict-
  // free with an odd number of 16-byte units per row); the two halves of a
  // warp cover the two halves of the columns of the same rows.
  {
    const int lane = gt & 31, w = gt >> 5;
    const int half = lane >> 4;
    const int h0 = (ncg + 1) >> 1;
    const int cg_begin = half ? h0 : 0, cg_end = half ? ncg : h0;
    for (int base = w * 16; base < dred; base += kWarps * 16) {
      const int red = base + (lane & 15);
      float o[NX];
#pragma unroll
      for (int c = 0; c < NX; ++c) o[c] = 0.f;
      if (red < dred) {
        const float *nrow = Nb + red * kpad;
        for (int cg0 = cg_begin; cg0 < cg_end; cg0 += 4) {
          float4 n4[4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            n4[u] = (cg0 + u < cg_end) ? *reinterpret_cast<const float4 *>(nrow + 4 * (cg0 + u))
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (cg0 + u < cg_end) {
#pragma unroll
              for (int c = 0; c < NX; ++c) {
                const float4 t4 = *reinterpret_cast<const float4 *>(G.t + c * kpad + 4 * (cg0 + u));
                o[c] = fmaf(n4[u].x, t4.x, o[c]);
                o[c] = fmaf(n4[u].y, t4.y, o[c]);
                o[c] = fmaf(n4[u].z, t4.z, o[c]);
                o[c] = fmaf(n4[u].w, t4.w, o[c]);
              }
            }
          }
        }
      }
#pragma unroll
      for (int c = 0; c < NX; ++c) o[c] += __shfl_xor_sync(0xffffffffu, o[c], 16);
      if (red < dred && half == 0) {
#pragma unroll
        for (int c = 0; c < NX; ++c) G.psired[c * ldr + red] = o[c] + q_p[c * it.dred_pad + red];
      }
    }
  }
  group_sync(g, GT);

  // slot-0 states pinned to e_c; Lambda-comp; residuals; new exchange sums
  float prim_f = 0.f, dual_f = 0.f;  // FP32 partials per thread and warp, combined in FP64
  for (int f = gt, mpos = mpos0, r = r0; f < dcol; f += GT, mpos += dm, r += dr) {
    if (r >= r_sub) { r -= r_sub; ++mpos; }
    const int red = mpos * rs_red + r - NX;
    const float a = alpha[f];
    float gsum = 0.f;
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      const float psi_old = psi_p[c * dcol + f];
      const float lam_old = lam_p[c * dcol + f];
      const float vv = psi_old + a * xj[c];
      const float ps = (r < NX) ? ((mpos == it.self_pos && r == c) ? 1.f : 0.f) : G.psired[c * ldr + red];
      const float lam_new = vv - ps;
      const float dp = lam_new - lam_old;
      const float dd = ps - psi_old;
      prim_f = fmaf(dp, dp, prim_f);
      dual_f = fmaf(dd, dd, dual_f);
      psi_p[c * dcol + f] = ps;
      lam_p[c * dcol + f] = lam_new;
      if (P.Phi) P.Phi[it.st_off + c * dcol + f] = lam_new - lam_old + ps;
      gsum = fmaf(2.f * ps - vv, xj[c], gsum);
    }
    Gnext[reinterpret_cast<const int *>(tab + mpos * MT)[3] + r] = gsum;
  }
  // GB300 runs FP64 at a small fraction of FP32: sums of a few squares stay in
  // FP32 (tree order, relative error ~1e-6), the per-warp sums are combined
  // in FP64 and Conv compares squared residuals (no square root on the path).
  const float prim_w = warp_sum_f(prim_f);
  const float dual_w = warp_sum_f(dual_f);
  if ((gt & 31) == 0) {
    G.red[2 * (gt >> 5)] = (double)prim_w;
    G.red[2 * (gt >> 5) + 1] = (double)dual_w;
  }
  group_sync(g, GT);
  if (gt == 0) {
    double pp = 0.0, dd = 0.0;
    for (int w = 0; w < kWarps; ++w) {
      pp += G.red[2 * w];
      dd += G.red[2 * w + 1];
    }
    const double epsp = extra[1], epsd = extra[2];
    const double rho2 = (double)rho * (double)rho;
    const bool conv = pp <= epsp * epsp && rho2 * dd <= epsd * epsd;
    const float rj = sqrtf((float)pp);
    const float sj = rho * sqrtf((float)dd);
    P.item_r[idx] = rj;
    P.item_s[idx] = sj;
    if (!(isfinite(rj) && isfinite(sj))) set_error(P.err, DLMPC_ERR_NONFINITE, blockIdx.x, iter, it.sub);
    if (!conv) atomicAdd(lnc + it.lslot, 1u);
  }
}

__device__ __forceinline__ void red_add_release_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// CTA-wide bounded barrier on the rotating 64-bit counter of barrier number e.
// Returns false on timeout or when any CTA has recorded an error; `total` is
// the number of not-converged patches summed over the grid.
__device__ __forceinline__ bool sweep_barrier(const Params &P, unsigned e, unsigned my_nc, unsigned long long *prev_hi,
                                              unsigned &total, int iter) {
  __shared__ int ok_sh;
  __shared__ unsigned total_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long *ctr = P.bar + (e % 3);
    red_add_release_u64(ctr, 1ull | ((unsigned long long)my_nc << 32));
    const unsigned target = (e / 3 + 1) * gridDim.x;
    const unsigned long long t0 = global_ns();
    int ok = 1;
    unsigned long long v = 0;
    for (unsigned spins = 0;; ++spins) {
      v = ld_acquire_u64(ctr);
      if ((unsigned)(v & 0xffffffffull) >= target) break;
      if ((spins & 63u) == 63u) {
        if (ld_volatile_i32(P.err) != 0) { ok = 0; break; }
        if (global_ns() - t0 > P.timeout_ns) {
          set_error(P.err, DLMPC_ERR_TIMEOUT, blockIdx.x, iter, 0);
          ok = 0;
          break;
        }
      }
    }
    if (ok && ld_volatile_i32(P.err) != 0) ok = 0;
    const unsigned long long hi = v >> 32;
    total_sh = (unsigned)(hi - prev_hi[e % 3]);
    prev_hi[e % 3] = hi;
    ok_sh = ok;
  }
  __syncthreads();
  total = total_sh;
  return ok_sh != 0;
}

template <int NX, int GT>
__global__ void __launch_bounds__(1024, 1) sweep_kernel(Params P) {
  extern __shared__ __align__(16) float sm[];
  const int tid = threadIdx.x;
  const int g = tid / GT, gt = tid - g * GT;
  const int b = blockIdx.x;
  const GroupLayout L = group_layout(NX, P.nu, GT, P.wave, P.max_dcol, P.max_dred_pad, P.max_kpad, P.max_nmem);
  float *gbase = sm + g * P.grp_floats;
  Group G;
  G.alpha = gbase + L.alpha;
  G.vred = gbase + L.vred;
  G.psired = gbase + L.psired;
  G.t = gbase + L.t;
  G.part = gbase + L.part;
  G.red = reinterpret_cast<double *>(gbase + L.red);
  G.mtab = gbase + L.mtab;
  G.icache = gbase + L.icache;
  G.mbar = reinterpret_cast<uint64_t *>(gbase + L.mbar);
  G.phase = 0;
  float *cta = sm + P.ng * P.grp_floats;
  unsigned long long *prev_hi = reinterpret_cast<unsigned long long *>(cta);  // [3] (+1 pad)
  unsigned *lnc = reinterpret_cast<unsigned *>(cta + 8);                      // [max_local_inst]
  int *lact = reinterpret_cast<int *>(cta + 8 + P.max_local_inst);            // [max_local_inst]
  float *arena = cta + P.cta_floats;

  const int gi0 = P.grp_ptr[b * P.ng + g];
  const int gi1 = P.grp_ptr[b * P.ng + g + 1];
  const int li0 = P.cta_inst_ptr[b], nli = P.cta_inst_ptr[b + 1] - li0;
  const bool one_wave = gi1 - gi0 <= P.wave;  // member tables filled once per launch

  if (gt == 0) mbar_init(G.mbar, 1);
  if (tid < 3) prev_hi[tid] = 0ull;
  __syncthreads();

  // ---- prologue: s_i, starting state, resident data, starting exchange sums
  bool ok = true;
  for (int ii = gi0; ii < gi1; ++ii) {
    const int idx = P.grp_items[ii];
    const Item it = P.items[idx];
    const int dcol = it.r_sub * it.n_mem;
    if (gt < 32) {
      double s = 0.0;
      for (int e = gt; e < it.n_mem * NX; e += 32) {
        const int m = P.members[it.mem_off + e / NX];
        const double xv = P.x[(int64_t)m * NX + (e % NX)];
        s += xv * xv;
      }
      s = warp_sum_d(s);
      if (gt == 0) P.S[it.sub] = (float)s;
    }
    float *psi_g = P.Psi + it.st_off, *lam_g = P.Lam + it.st_off;
    float *psi_p = it.st_sm >= 0 ? arena + it.st_sm : psi_g;
    float *lam_p = it.st_sm >= 0 ? arena + it.st_sm + NX * dcol : lam_g;
    for (int e = gt; e < NX * dcol; e += GT) {
      const float ps = (P.warm == DLMPC_WARM_COLD) ? 0.f : psi_g[e];
      const float lm = (P.warm == DLMPC_WARM_COLD) ? 0.f : lam_g[e];
      psi_p[e] = ps;
      lam_p[e] = lm;
    }
    if (it.q_sm >= 0)
      for (int e = gt; e < NX * it.dred_pad; e += GT) arena[it.q_sm + e] = P.qvec[it.q_off + e];
    if (it.n_sm >= 0) {
      if (gt == 0) tma_load_1d(arena + it.n_sm, P.Nmat + it.n_off, (unsigned)it.dred_pad * it.kpad * 4u, G.mbar);
      ok = mbar_wait(G.mbar, G.phase & 1u, P.timeout_ns) && ok;
      ++G.phase;
    }
    group_sync(g, GT);
    float xj[NX];
#pragma unroll
    for (int c = 0; c < NX; ++c) xj[c] = P.x[(int64_t)it.sub * NX + c];
    const int *mem = P.members + it.mem_off;
    const int *rev = P.rev_slot + it.mem_off;
    for (int f = gt; f < dcol; f += GT) {
      const int mpos = f / it.r_sub, r = f - mpos * it.r_sub;
      float gsum = 0.f;
#pragma unroll
      for (int c = 0; c < NX; ++c) gsum = fmaf(psi_p[c * dcol + f] - lam_p[c * dcol + f], xj[c], gsum);
      P.G0[P.g_off[mem[mpos]] + (int64_t)rev[mpos] * it.r_sub + r] = gsum;
    }
  }
  if (!ok && gt == 0) set_error(P.err, DLMPC_ERR_TIMEOUT, b, -1, 2);
  if (b == 0) {
    for (int e = tid; e < 3 * P.n_inst; e += blockDim.x) P.notconv[e] = 0u;
    for (int e = tid; e < P.n_inst; e += blockDim.x) P.inst_iters[e] = 0;
  }
  unsigned total = 0;
  unsigned e_bar = 0;
  ok = sweep_barrier(P, e_bar++, 0u, prev_hi, total, -1);
  // s_m of every member is now visible: single-wave groups fill their tables once
  if (ok && one_wave && gi1 > gi0) {
    fill_wave<NX>(P, P.grp_items + gi0, gi1 - gi0, G.icache, G.mtab, gt, GT);
    group_sync(g, GT);
  }

  // ---- ADMM iterations (Alg. 2)
  const int n_it = P.fixed_iters > 0 ? P.fixed_iters : P.max_iter;
  const bool multi = P.n_inst > 1;
  const int MT = member_record(NX, P.nu);
  int iter = 0;
  for (; ok && iter < n_it; ++iter) {
    const int slot = iter % 3, prev = (iter + 2) % 3;
    if (b == 0 && multi)
      for (int e = tid; e < P.n_inst; e += blockDim.x) P.notconv[((iter + 1) % 3) * P.n_inst + e] = 0u;
    for (int t = tid; t < nli; t += blockDim.x) {
      lnc[t] = 0u;
      int active = 1;
      if (multi && P.fixed_iters <= 0 && iter > 0)
        active = ld_acquire_u32(P.notconv + prev * P.n_inst + P.cta_inst[li0 + t]) > 0u;
      lact[t] = active;
    }
    __syncthreads();
    trace_point(P, iter, 0);
    const float *Gcur = (iter & 1) ? P.G1 : P.G0;
    float *Gnext = (iter & 1) ? P.G0 : P.G1;
    for (int w0 = gi0; w0 < gi1; w0 += P.wave) {
      const int wn = min(P.wave, gi1 - w0);
      if (!one_wave) {
        group_sync(g, GT);  // the previous wave is done with the cache
        fill_wave<NX>(P, P.grp_items + w0, wn, G.icache, G.mtab, gt, GT);
        group_sync(g, GT);
      }
      for (int wi = 0; wi < wn; ++wi) {
        const Item &it = cached_item(G.icache, wi);
        if (!lact[it.lslot]) continue;
        phi_rows<NX, GT>(P, it, G.mtab + wi * P.max_nmem * MT, Gcur, G.alpha + wi * P.max_dcol,
                         cached_extra(G.icache, wi)[0], gt);
      }
      group_sync(g, GT);
      if (w0 == gi0) trace_point(P, iter, 1);
      for (int wi = 0; wi < wn; ++wi) {
        const Item &it = cached_item(G.icache, wi);
        if (!lact[it.lslot]) continue;
        const float *ex = cached_extra(G.icache, wi);
        project_item<NX, GT>(P, reinterpret_cast<const int *>(ex)[3], it, G.mtab + wi * P.max_nmem * MT, ex, G,
                             G.alpha + wi * P.max_dcol, arena, Gnext, g, gt, lnc, iter, w0 == gi0 && wi == 0);
        if (w0 == gi0 && wi == 0) trace_point(P, iter, 2);
      }
      group_sync(g, GT);
    }
    trace_point(P, iter, 3);
    __syncthreads();
    trace_point(P, iter, 4);
    if (b == P.skip_arrival_cta) {  // test only: never arrive, the others' waits run out
      ok = false;
      break;
    }
    unsigned my_nc = 0;
    if (tid == 0) {
      for (int t = 0; t < nli; ++t) {
        my_nc += lnc[t];
        if (multi && lnc[t]) atomicAdd(P.notconv + slot * P.n_inst + P.cta_inst[li0 + t], lnc[t]);
      }
    }
    ok = sweep_barrier(P, e_bar++, my_nc, prev_hi, total, iter);
    if (!ok) break;
    trace_point(P, iter, 5);
    if (b == 0) {
      if (multi) {
        for (int e = tid; e < P.n_inst; e += blockDim.x)
          if (P.inst_iters[e] == 0 && ld_acquire_u32(P.notconv + slot * P.n_inst + e) == 0u) P.inst_iters[e] = iter + 1;
      } else if (tid == 0 && total == 0u && P.inst_iters[0] == 0) {
        P.inst_iters[0] = iter + 1;
      }
    }
    if (P.fixed_iters <= 0 && total == 0u) { ++iter; break; }
  }
  if (b == 0 && tid == 0) P.err[4] = iter;

  // ---- epilogue: write back resident state, dynamics
  __syncthreads();
  for (int ii = gi0; ii < gi1; ++ii) {
    const Item &it = P.items[P.grp_items[ii]];
    if (it.st_sm < 0) continue;
    const int n2 = 2 * NX * it.r_sub * it.n_mem;
    const int half = n2 / 2;
    for (int e = gt; e < n2; e += GT) {
      const float v = arena[it.st_sm + e];
      if (e < half) P.Psi[it.st_off + e] = v;
      else P.Lam[it.st_off + e - half] = v;
    }
  }
  if (ok && P.x_next) {
    for (int ii = gi0; ii < gi1; ++ii) {
      const Item &it = P.items[P.grp_items[ii]];
      const int j = it.sub;
      if (gt < NX) {
        const int a = gt;
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
  __syncthreads();
  if (gt == 0) mbar_inval(G.mbar);
}

// ---------------------------------------------------------------------------
// host-side launch helpers
// ---------------------------------------------------------------------------

template <int NX, int GT>
static const void *sweep_fn() {
  return reinterpret_cast<const void *>(&sweep_kernel<NX, GT>);
}

const void *sweep_kernel_ptr(int nx, int gt) {
#define DLMPC_SWEEP_CASE(NXV)                    \
  case NXV:                                      \
    if (gt == 64) return sweep_fn<NXV, 64>();    \
    if (gt == 128) return sweep_fn<NXV, 128>();  \
    if (gt == 256) return sweep_fn<NXV, 256>();  \
    return nullptr;
  switch (nx) {
    DLMPC_SWEEP_CASE(1)
    DLMPC_SWEEP_CASE(2)
    DLMPC_SWEEP_CASE(3)
    DLMPC_SWEEP_CASE(4)
  }
#undef DLMPC_SWEEP_CASE
  return nullptr;
}

int sweep_group_floats(int nx, int nu, int gt, int wave, int max_dcol, int max_dred_pad, int max_kpad, int max_nmem) {
  return group_layout(nx, nu, gt, wave, max_dcol, max_dred_pad, max_kpad, max_nmem).total;
}

cudaError_t launch_sweep(const Params &P, int gt, int grid, size_t smem, cudaStream_t s) {
  const void *fn = sweep_kernel_ptr(P.nx, gt);
  if (!fn) return cudaErrorInvalidValue;
  Params pc = P;
  void *args[] = {&pc};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(gt * P.ng);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace dlmpc
