// Persistent ADMM sweep for sm_103a: one cooperative launch per MPC step runs
// the per-step precompute, every iteration of Alg. 2 (Phi-comp, Psi-comp,
// Lambda-comp, Conv) and the dynamics of Alg. 1.
//
// Work split.  One CTA per SM; the CTA is cut into `ng` independent groups of
// GT threads that synchronise with named barriers.  Every column patch
// ("item", Sec. III-D) belongs to one group.  A group handles its items in
// waves: the Phi-step scalars of every row of the wave's patches first (all
// exchange loads of the wave in flight together), then per item Psi-comp,
// Lambda-comp and the residuals.  The first iteration of a step projects the
// stored Psi and Lambda (project_item: psi = q + N (N^T v)); the later ones run
// on the compact iterate (project_compact), and the final Psi and Lambda are
// formed once at the end (expand_compact).
//
// Shared memory.  Per group: the Phi-step scalars, work vectors, per-warp
// partial sums, a record per patch member and one per patch row (exchange
// offsets, |Patch|, weights, bounds, 1/s, cost blocks) so the Phi-step issues
// only the exchange loads.  After the groups: per-CTA counters, then the
// items' resident data placed by the host: the compact iterate, N (loaded
// once per launch by a 1-D bulk TMA copy) where room remains, then Psi,
// Lambda and q.  N of the other patches, and N^T of every patch, are read
// from L2 in whole 16-byte units.
//
// Iteration barrier.  Each CTA adds (1 + not_converged << 32) to one of three
// rotating 64-bit counters with a release reduction: the low half counts
// arrivals, the high half sums the not-converged patches, so the global Conv
// decision needs no extra atomic or barrier.  Every wait is bounded.
//
// Variants.  The block instantiation (BLK) solves the Phi-step per (member,
// time slot) for full cost blocks, over the slot's box (slot_box_qp) or, with
// coupled rows, by the explicit solution that the prologue rebuilds for this
// x(tau) (build_region, slot_explicit).  Simulated lost messages (send) keep
// the receiver's last row sums in place of a fresh exchange value.
#pragma once
#include <cuda_runtime.h>
#include <cmath>
#include <cstdint>

#include "dlmpc_common.cuh"
#include "dlmpc_internal.h"

namespace dlmpc {

struct GroupLayout {
  int alpha, vred, psired, t, part, red, mtab, rtab, icache, mbar, total;
};

// Floats of one cached item: the Item, then rho, eps_p, eps_d, its own index.
constexpr int kItemFloats = (int)((sizeof(Item) + 3) / 4) + 4;

__host__ __device__ inline int round4(int v) { return (v + 3) & ~3; }
__host__ __device__ inline int max3(int a, int b, int c) { return a > b ? (a > c ? a : c) : (b > c ? b : c); }

// Floats of one patch-member record: exchange read offset, |Patch|, 1/s (0
// when s = 0), exchange write base, then x[nx], rho/(rho + 2 q s)[nx],
// x_lo[nx], x_hi[nx], rho/(rho + 2 r s)[nu], u_lo[nu], u_hi[nu], 2 Q_m
// [nx][nx], 2 R_m [nu][nu].
__host__ __device__ inline int member_record(int nx, int nu) { return 4 + 4 * nx + 3 * nu + nx * nx + nu * nu; }

// Floats of one cached row record (RowRec: four ints, four floats).
constexpr int kRowRecord = 8;

// Float offsets inside one group region; the host uses the same function.
// rows_cached: the plan keeps one record per patch row (row_rec) in shared
// memory, filled once per launch -- plans whose groups hold one wave of items;
// other plans derive the records where they are used.
__host__ __device__ inline GroupLayout group_layout(int nx, int nu, int gt, int wave, int max_dcol, int max_dred_pad,
                                                    int max_kpad, int max_nmem, bool rows_cached) {
  GroupLayout L;
  int o = 0;
  L.alpha = o;  o += round4(wave * max_dcol);
  L.vred = o;   o += nx * max_dred_pad;
  L.psired = L.vred;  // psi_red is written only after the last read of v_red
  L.t = o;      o += round4(nx * max_kpad);
  L.part = o;   o += round4(max3((gt / 32) * nx * max_kpad, 4 * gt, max_dred_pad));
  L.red = o;    o += round4(4 * (gt / 32));
  L.mtab = o;   o += round4(wave * max_nmem * member_record(nx, nu));
  L.rtab = o;   o += rows_cached ? wave * max_dcol * kRowRecord : 0;
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
  float *alpha, *vred, *psired, *t, *part, *mtab, *rtab, *icache;
  float *red;
  uint64_t *mbar;
  unsigned phase;  // completed bulk copies on mbar
};

// Record of row p of a patch (reduced order: the reduced rows, then the
// slot-0 rows), from its member's record `tab`: exchange read offset,
// |Patch(m)|, exchange write offset, aux (u index sub * nu + b of an own
// slot-0 input row, own state index c of an own slot-0 state row, else -1);
// den = rho / (rho + 2 q s), the row's bounds (slot-0 state rows unbounded),
// 1/s (0 when s = 0).
struct RowRec {
  int rd, np, wr, aux;
  float den, lo, hi, inv_s;
};

template <int NX>
__device__ __forceinline__ RowRec row_rec(const Params &P, const Item &it, const float *tab, int p) {
  const int MT = member_record(NX, P.nu);
  const int rs_red = it.r_sub - NX, dred = it.dred, nxT = NX * it.T;
  int mpos, r;
  if (p < dred) {
    mpos = small_div(p, rs_red);
    r = p - mpos * rs_red + NX;
  } else {
    mpos = small_div(p - dred, NX);
    r = p - dred - mpos * NX;
  }
  const float *rec = tab + mpos * MT;
  const int *reci = reinterpret_cast<const int *>(rec);
  const bool own = mpos == it.self_pos;
  RowRec o;
  o.aux = -1;
  if (r < nxT) {
    const int a = r % NX;
    o.den = rec[4 + NX + a];
    o.lo = r >= NX ? rec[4 + 2 * NX + a] : -INFINITY;
    o.hi = r >= NX ? rec[4 + 3 * NX + a] : INFINITY;
    if (own && r < NX) o.aux = r;
  } else {
    const int bb = (r - nxT) % P.nu;
    o.den = rec[4 + 4 * NX + bb];
    o.lo = rec[4 + 4 * NX + P.nu + bb];
    o.hi = rec[4 + 4 * NX + 2 * P.nu + bb];
    if (own && r < nxT + P.nu) o.aux = it.sub * P.nu + bb;
  }
  o.rd = reci[0] + r;
  o.np = reci[1];
  o.wr = reci[3] + r;
  o.inv_s = rec[2];
  return o;
}

// Caches the wave's items (with their instance constants) and fills the member
// records of their patches, so the iteration loop reads nothing but the
// exchange sums (and non-resident N) from global memory; with cached rows
// (P.rows_cached) also the record of every patch row (row_rec), else each
// row's record is derived from its member's where it is used.
template <int NX>
__device__ __forceinline__ void fill_wave(const Params &P, const int *items, int wn, float *icache, float *mtab,
                                          float *rtab, int g, int gt, int GT) {
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
      float *blk = rec + 4 + 4 * NX + 3 * P.nu;
      for (int e2 = 0; e2 < NX * NX; ++e2) blk[e2] = P.qblk2[(int64_t)m * NX * NX + e2];
      for (int e2 = 0; e2 < P.nu * P.nu; ++e2) blk[NX * NX + e2] = P.rblk2[(int64_t)m * P.nu * P.nu + e2];
    }
  }
  if (!P.rows_cached) return;
  group_sync(g, GT);  // the member records are complete
  for (int wi = 0; wi < wn; ++wi) {
    const Item &it = P.items[items[wi]];
    const float *tab = mtab + wi * P.max_nmem * MT;
    float *rt = rtab + wi * P.max_dcol * kRowRecord;
    for (int p = gt; p < it.r_sub * it.n_mem; p += GT) {
      const RowRec r = row_rec<NX>(P, it, tab, p);
      *reinterpret_cast<int4 *>(rt + p * kRowRecord) = make_int4(r.rd, r.np, r.wr, r.aux);
      *reinterpret_cast<float4 *>(rt + p * kRowRecord + 4) = make_float4(r.den, r.lo, r.hi, r.inv_s);
    }
  }
}

// The cached record of row p.
__device__ __forceinline__ RowRec cached_row(const float *rt, int p) {
  const int4 a = *reinterpret_cast<const int4 *>(rt + p * kRowRecord);
  const float4 c = *reinterpret_cast<const float4 *>(rt + p * kRowRecord + 4);
  RowRec r;
  r.rd = a.x;
  r.np = a.y;
  r.wr = a.z;
  r.aux = a.w;
  r.den = c.x;
  r.lo = c.y;
  r.hi = c.z;
  r.inv_s = c.w;
  return r;
}

// The record of row p: cached (rows_cached plans), else derived.
template <int NX>
__device__ __forceinline__ RowRec get_row(const Params &P, const Item &it, const float *tab, const float *rt, int p) {
  return P.rows_cached ? cached_row(rt, p) : row_rec<NX>(P, it, tab, p);
}

__device__ __forceinline__ const Item &cached_item(const float *icache, int wi) {
  return *reinterpret_cast<const Item *>(icache + wi * kItemFloats);
}
__device__ __forceinline__ const float *cached_extra(const float *icache, int wi) {
  return icache + wi * kItemFloats + (int)((sizeof(Item) + 3) / 4);
}


// Simulated lost messages (the fully distributed setting, Sec. V): output n
// of SplitMix64 (Steele, Lea and Flood, 2014) seeded with `seed` ...
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t n) {
  uint64_t z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ... decides whether the row sums patch j sends to member m = *mp at the end
// of iteration k are lost: draw n = (k N + j) N + m, lost when its top 53 bits
// are below the threshold floor(p 2^53).  A lost message leaves the value the
// receiver holds, so the writer copies the slot's current value forward.  The
// member is read only when messages can be lost.
__device__ __forceinline__ float send(const Params &P, int iter, int j, const int *mp, int idx, float fresh) {
  if (P.stale_thr == 0ull) return fresh;
  const int m = *mp;
  const uint64_t N = (uint64_t)P.n_items;
  const uint64_t n = ((uint64_t)iter * N + (uint64_t)j) * N + (uint64_t)m;
  const float *Gcur = (iter & 1) ? P.G1 : P.G0;  // read this iteration, the receiver's value
  return (splitmix64_at(P.stale_seed, n) >> 11) < P.stale_thr ? __ldcg(Gcur + idx) : fresh;
}

// Closed form of one row from its w and row record (see phi_rows).
__device__ __forceinline__ void phi_row(const Params &P, int p, int dred, int aux, float4 c, float w,
                                        float *alpha_out) {
  // z* = rho w / (rho + 2 q s), clipped; alpha = (z - w) / s; s = 0 gives phi = v
  float al = 0.f, z = w;
  if (c.w > 0.f) {
    z = fminf(fmaxf(w * c.x, c.y), c.z);
    al = (z - w) * c.w;
  }
  alpha_out[p] = al;
  if (aux >= 0 && p < dred) P.u[aux] = z;
}

// Phi-comp for every row of one patch (Sec. II-A row problem, closed form):
// w = (Psi - Lambda)_r . x_hat from the exchange sums, z = clip(rho w / (rho +
// 2 q s), lo, hi), alpha = (z - w) / s (0 when s = 0).  The new Phi row is
// Psi_r - Lambda_r + alpha x_hat; only alpha is stored, in reduced order
// (the reduced rows, then the slot-0 rows).  A thread takes two rows at a
// time and issues the exchange loads of both before adding them.
// W_ONLY: store w itself (the block Phi-step solves the slots afterwards).
template <int NX, int GT, bool W_ONLY, bool CACHED>
__device__ __forceinline__ void phi_rows(const Params &P, const Item &it, const float *tab, const float *rt,
                                         const float *Gcur, float *alpha_out, int gt) {
  const int r_sub = it.r_sub;
  const int dcol = r_sub * it.n_mem;
  for (int p = gt; p < dcol; p += 2 * GT) {
    const int p2 = p + GT;
    const bool two = p2 < dcol;
    const RowRec ra = CACHED ? cached_row(rt, p) : row_rec<NX>(P, it, tab, p);
    const int4 ia = make_int4(ra.rd, ra.np, ra.wr, ra.aux);
    const float4 ca = make_float4(ra.den, ra.lo, ra.hi, ra.inv_s);
    int4 ib = make_int4(0, 0, 0, -1);
    float4 cb = make_float4(0.f, 0.f, 0.f, 0.f);
    if (two) {
      const RowRec rb = CACHED ? cached_row(rt, p2) : row_rec<NX>(P, it, tab, p2);
      ib = make_int4(rb.rd, rb.np, rb.wr, rb.aux);
      cb = make_float4(rb.den, rb.lo, rb.hi, rb.inv_s);
    }
    const float *gp = Gcur + ia.x;
    const float *gp2 = Gcur + ib.x;
    float w = 0.f, w2 = 0.f;
    for (int s0 = 0; s0 < max(ia.y, ib.y); s0 += 8) {
      float gv[8], gv2[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        gv[j] = (s0 + j < ia.y) ? __ldcg(gp + (s0 + j) * r_sub) : 0.f;
        gv2[j] = (s0 + j < ib.y) ? __ldcg(gp2 + (s0 + j) * r_sub) : 0.f;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        w += gv[j];
        w2 += gv2[j];
      }
    }
    if constexpr (W_ONLY) {
      alpha_out[p] = w;
      if (two) alpha_out[p2] = w2;
    } else {
      phi_row(P, p, it.dred, ia.w, ca, w, alpha_out);
      if (two) phi_row(P, p2, it.dred, ib.w, cb, w2, alpha_out);
    }
  }
}

constexpr int kMaxQP = 4;

// argmin 1/2 z^T (C + cd I) z - cd w^T z  s.t.  lo <= z <= hi  (N <= kMaxQP,
// C symmetric positive semi-definite, cd > 0): every component free, at lo or
// at hi (finite bounds only).  A pattern's candidate solves the N x N system
// whose free rows are those of C + cd I (right-hand side cd w) and whose fixed
// rows are z_a = bound, by elimination without pivoting (the fixed rows are
// unit rows and the free pivots are Schur complements of a positive definite
// matrix).  The first feasible candidate whose gradient has the KKT signs on
// its fixed components is the optimum; should rounding let none pass, the
// feasible candidate of least objective is taken (the optimum of a strictly
// convex QP is one of them, and no feasible point is lower).
template <int N>
__device__ __forceinline__ void slot_box_qp(const float *C, float cd, const float (&w)[N], const float (&lo)[N],
                                            const float (&hi)[N], float (&z_out)[N]) {
  constexpr int kPat = N == 1 ? 3 : N == 2 ? 9 : N == 3 ? 27 : 81;
  float best = INFINITY;
#pragma unroll 1
  for (int pat = 0; pat < kPat; ++pat) {
    int d[N];
    bool ok = true;
    int rem = pat;
#pragma unroll
    for (int a = 0; a < N; ++a) {
      d[a] = rem % 3;
      rem /= 3;
      if ((d[a] == 1 && !(lo[a] > -INFINITY)) || (d[a] == 2 && !(hi[a] < INFINITY))) ok = false;
    }
    if (!ok) continue;
    float M[N][N + 1];
#pragma unroll
    for (int a = 0; a < N; ++a) {
#pragma unroll
      for (int c = 0; c < N; ++c)
        M[a][c] = d[a] == 0 ? C[a * N + c] + (a == c ? cd : 0.f) : (a == c ? 1.f : 0.f);
      M[a][N] = d[a] == 0 ? cd * w[a] : (d[a] == 1 ? lo[a] : hi[a]);
    }
#pragma unroll
    for (int q = 0; q < N; ++q) {
      const float inv = 1.f / M[q][q];
#pragma unroll
      for (int r = q + 1; r < N; ++r) {
        const float f = M[r][q] * inv;
#pragma unroll
        for (int c = q; c <= N; ++c) M[r][c] -= f * M[q][c];
      }
    }
    float z[N];
#pragma unroll
    for (int a = N - 1; a >= 0; --a) {
      float v = M[a][N];
#pragma unroll
      for (int c = a + 1; c < N; ++c) v -= M[a][c] * z[c];
      z[a] = v / M[a][a];
    }
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const float tol_lo = 1e-5f * fmaxf(1.f, fabsf(lo[a])), tol_hi = 1e-5f * fmaxf(1.f, fabsf(hi[a]));
      if (z[a] < lo[a] - tol_lo || z[a] > hi[a] + tol_hi) ok = false;
      z[a] = fminf(fmaxf(z[a], lo[a]), hi[a]);
    }
    if (!ok) continue;
    // KKT signs of the gradient g = H z - cd w on the fixed components
    // (g >= 0 at lo, g <= 0 at hi, to a relative 1e-5): the optimum at once
    bool kkt = true;
    float obj = 0.f;
#pragma unroll
    for (int a = 0; a < N; ++a) {
      float hz = cd * z[a], mag = fabsf(cd * z[a]) + fabsf(cd * w[a]);
#pragma unroll
      for (int c = 0; c < N; ++c) {
        hz = fmaf(C[a * N + c], z[c], hz);
        mag = fmaf(fabsf(C[a * N + c]), fabsf(z[c]), mag);
      }
      const float g = hz - cd * w[a], tol = 1e-5f * mag;
      if ((d[a] == 1 && g < -tol) || (d[a] == 2 && g > tol)) kkt = false;
      obj = fmaf(z[a], 0.5f * hz - cd * w[a], obj);
    }
    if (kkt) {
#pragma unroll
      for (int a = 0; a < N; ++a) z_out[a] = z[a];
      return;
    }
    if (obj < best) {
      best = obj;
#pragma unroll
      for (int a = 0; a < N; ++a) z_out[a] = z[a];
    }
  }
}

// In-place inverse of a symmetric positive definite matrix of order k <= N,
// Gauss-Jordan elimination without pivoting (the pivots of an SPD matrix are
// positive).
template <int N>
__device__ __forceinline__ void spd_inverse(float (&M)[N][N], int k) {
#pragma unroll
  for (int p = 0; p < N; ++p) {
    if (p < k) {
      const float inv = 1.f / M[p][p];
      M[p][p] = 1.f;
#pragma unroll
      for (int j = 0; j < N; ++j) M[p][j] *= inv;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        if (i != p && i < k) {
          const float f = M[i][p];
          M[i][p] = 0.f;
#pragma unroll
          for (int j = 0; j < N; ++j) M[i][j] -= f * M[p][j];
        }
      }
    }
  }
}

// Explicit solution of the slot QP, one region (Alg. 1: precomputed from x(tau)
// once per MPC step).  For the slot QP min 1/2 z^T H z - cd w^T z subject to
// its rows A z <= b, H = C + cd I (C = 2 Q_i or 2 R_i, cd = rho / s_i), the
// minimiser on the region's active rows {A_S z = b_S} and its multipliers are
// affine in w:
//   z  = K w + k,   K = cd (Hi - P M^{-1} P^T),  k = P M^{-1} b_S,
//   mu = L w + l,   L = cd M^{-1} P^T,           l = -M^{-1} b_S,
// with Hi = H^{-1}, P = Hi A_S^T (N x |S|) and M = A_S P (|S| x |S|, SPD since
// the rows of A_S are independent).  Writes K [N][N], k [N], L [N][N] (rows
// below |S| used), l [N].
template <int N>
__device__ void build_region(const Params &P, int sub, int kind, int r, float cd) {
  const int key = 2 * sub + kind;
  const float *C = kind == 0 ? P.qblk2 + (int64_t)sub * N * N : P.rblk2 + (int64_t)sub * N * N;
  const uint32_t desc = P.rg_desc[P.rg_base[key] + r];
  const int k = desc & 15u;
  const int cs = P.crow_stride;
  const float *rows = P.crow + (int64_t)P.rw_base[key] * cs;
  float Hi[N][N], Pm[N][N], M[N][N], bs[N];
#pragma unroll
  for (int a = 0; a < N; ++a)
#pragma unroll
    for (int c = 0; c < N; ++c) Hi[a][c] = C[a * N + c] + (a == c ? cd : 0.f);
  spd_inverse<N>(Hi, N);
  // P = Hi A_S^T, b_S
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const float *aj = rows + (int)((desc >> (4 + 4 * j)) & 15u) * cs;
    bs[j] = j < k ? aj[cs - 1] : 0.f;
#pragma unroll
    for (int a = 0; a < N; ++a) {
      float v = 0.f;
      if (j < k)
#pragma unroll
        for (int c = 0; c < N; ++c) v = fmaf(Hi[a][c], aj[c], v);
      Pm[a][j] = v;
    }
  }
  // M = A_S P, inverted
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float *ai = rows + (int)((desc >> (4 + 4 * i)) & 15u) * cs;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float v = 0.f;
      if (i < k && j < k)
#pragma unroll
        for (int c = 0; c < N; ++c) v = fmaf(ai[c], Pm[c][j], v);
      M[i][j] = v;
    }
  }
  spd_inverse<N>(M, k);
  // Q = M^{-1} P^T (|S| x N): the multiplier map over cd
  float Qm[N][N];
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int c = 0; c < N; ++c) {
      float v = 0.f;
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (i < k && j < k) v = fmaf(M[j][i], Pm[c][i], v);
      Qm[j][c] = v;
    }
  float *out = P.expl + (int64_t)(P.rg_base[key] + r) * P.expl_stride;
#pragma unroll
  for (int a = 0; a < N; ++a) {
    // (P M^{-1})[a][j] = Qm[j][a] (M^{-1} is symmetric)
    float kk = 0.f, lj = 0.f;
#pragma unroll
    for (int j = 0; j < N; ++j) kk = fmaf(Qm[j][a], bs[j], kk);
#pragma unroll
    for (int c = 0; c < N; ++c) {
      float v = Hi[a][c];
#pragma unroll
      for (int j = 0; j < N; ++j) v -= Qm[j][a] * Pm[c][j];
      out[a * N + c] = cd * v;
      out[N * N + N + a * N + c] = cd * Qm[a][c];
    }
#pragma unroll
    for (int i = 0; i < N; ++i) lj = fmaf(M[a][i], bs[i], lj);
    out[N * N + a] = kk;
    out[2 * N * N + N + a] = -lj;
  }
}

// Evaluates the explicit solution of one slot, region by region in the
// order of the setup (active sets by size, the empty one first): the first
// region whose minimiser z = K w + k satisfies every row of the slot and whose
// multipliers mu = L w + l are non-negative (both to a relative 1e-5) is the
// optimum.  Should rounding let none pass, the feasible region of least
// objective 1/2 z^T H z - cd w^T z is taken (the optimum of a strictly convex
// QP is the minimiser on its own active rows, and no feasible point is lower).
// The slot-0 state has the empty region only.
template <int N>
__device__ __forceinline__ void slot_explicit(const Params &P, int key, bool slot0, const float *C, float cd,
                                              const float (&w)[N], float (&z_out)[N]) {
  const int nreg = slot0 ? 1 : P.rg_cnt[key];
  const int nrow = slot0 ? 0 : P.rw_cnt[key];
  const int cs = P.crow_stride;
  const int base = P.rg_base[key];
  const float *tb = P.expl + (int64_t)base * P.expl_stride;
  const float *rows = P.crow + (int64_t)P.rw_base[key] * cs;
  float best = INFINITY;
#pragma unroll 1
  for (int r = 0; r < nreg; ++r, tb += P.expl_stride) {
    float z[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
      float v = __ldcg(tb + N * N + a);
#pragma unroll
      for (int c = 0; c < N; ++c) v = fmaf(__ldcg(tb + a * N + c), w[c], v);
      z[a] = v;
    }
    bool ok = true;
    for (int j = 0; j < nrow; ++j) {
      const float *aj = rows + j * cs;
      float v = 0.f;
#pragma unroll
      for (int c = 0; c < N; ++c) v = fmaf(aj[c], z[c], v);
      const float bj = aj[cs - 1];
      if (v > bj + 1e-5f * fmaxf(1.f, fabsf(bj))) ok = false;
    }
    if (!ok) continue;
    const int k = r == 0 ? 0 : (int)(P.rg_desc[base + r] & 15u);
    bool dual = true;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      if (j < k) {
        const float lj = __ldcg(tb + 2 * N * N + N + j);
        float mu = lj, mag = fabsf(lj);
#pragma unroll
        for (int c = 0; c < N; ++c) {
          const float t = __ldcg(tb + N * N + N + j * N + c) * w[c];
          mu += t;
          mag += fabsf(t);
        }
        if (mu < -1e-5f * mag) dual = false;
      }
    }
    if (dual) {
#pragma unroll
      for (int a = 0; a < N; ++a) z_out[a] = z[a];
      return;
    }
    float obj = 0.f;
#pragma unroll
    for (int a = 0; a < N; ++a) {
      float hz = cd * z[a];
#pragma unroll
      for (int c = 0; c < N; ++c) hz = fmaf(C[a * N + c], z[c], hz);
      obj = fmaf(z[a], 0.5f * hz - cd * w[a], obj);
    }
    if (obj < best) {
      best = obj;
#pragma unroll
      for (int a = 0; a < N; ++a) z_out[a] = z[a];
    }
  }
}

// One slot of the block Phi-step: its N rows start at reduced position p0 and
// hold w (from the row pass) in alpha; the slot QP gives z, and alpha becomes
// (z - w)/s per row (0 when s = 0); own slot-0 inputs also give u(tau).
template <int N, int NX>
__device__ __forceinline__ void slot_solve(const Params &P, int key, bool slot0, int p0, int dred, const float *rec,
                                           const float *C, const Item &it, const float *tab, const float *rt,
                                           float *alpha, float rho) {
  float w[N], lo[N], hi[N], z[N];
  int aux[N];
#pragma unroll
  for (int a = 0; a < N; ++a) {
    const int p = p0 + a;
    const RowRec rr = get_row<NX>(P, it, tab, rt, p);
    w[a] = alpha[p];
    aux[a] = rr.aux;
    lo[a] = rr.lo;
    hi[a] = rr.hi;
    z[a] = w[a];
  }
  const float inv_s = rec[2];
  if (inv_s > 0.f) {
    if (P.expl)
      slot_explicit<N>(P, key, slot0, C, rho * inv_s, w, z);
    else
      slot_box_qp<N>(C, rho * inv_s, w, lo, hi, z);
  }
#pragma unroll
  for (int a = 0; a < N; ++a) {
    const int p = p0 + a;
    alpha[p] = inv_s > 0.f ? (z[a] - w[a]) * inv_s : 0.f;
    if (aux[a] >= 0 && p < dred) P.u[aux[a]] = z[a];
  }
}

// Phi-comp with full cost blocks Q_i, R_i: the rows of one member at one time
// slot (its nx state rows or its nu input rows, consecutive in reduced order)
// share x_hat and are solved together.  The row pass (phi_rows with W_ONLY)
// has left w per row in alpha; here one thread per slot solves
// min z^T C z + rho/(2 s) ||z - w||^2 over the slot's box (slot_box_qp with
// H = 2 C + (rho/s) I) or, with coupled rows, over the slot's polytope
// (slot_explicit), and alpha = (z - w)/s per row.
template <int NX>
__device__ void phi_slots(const Params &P, const Item &it, const float *tab, const float *rt, float *alpha,
                          float rho, int gt, int GT) {
  const int T = it.T, rs_red = it.r_sub - NX, dred = it.dred, nu = P.nu;
  const int MT = member_record(NX, nu);
  // the state slots of every member first, then the input slots: the costly
  // state slots share the first round over the group's threads
  const int nst = it.n_mem * T;
  for (int g = gt; g < it.n_mem * (2 * T - 1); g += GT) {
    int mpos, kk;
    if (g < nst) {
      mpos = small_div(g, T);
      kk = g - mpos * T;
    } else {
      mpos = small_div(g - nst, T - 1);
      kk = T + (g - nst - mpos * (T - 1));
    }
    const float *rec = tab + mpos * MT;
    const float *C = rec + 4 + 4 * NX + 3 * nu;
    const int key = P.expl ? 2 * P.members[it.mem_off + mpos] : 0;
    if (kk < T) {
      const int p0 = kk == 0 ? dred + mpos * NX : mpos * rs_red + (kk - 1) * NX;
      slot_solve<NX, NX>(P, key, kk == 0, p0, dred, rec, C, it, tab, rt, alpha, rho);
    } else {
      const int p0 = mpos * rs_red + (T - 1) * NX + (kk - T) * nu;
      C += NX * NX;
      switch (nu) {
        case 1: slot_solve<1, NX>(P, key + 1, false, p0, dred, rec, C, it, tab, rt, alpha, rho); break;
        case 2: slot_solve<2, NX>(P, key + 1, false, p0, dred, rec, C, it, tab, rt, alpha, rho); break;
        case 3: slot_solve<3, NX>(P, key + 1, false, p0, dred, rec, C, it, tab, rt, alpha, rho); break;
        default: slot_solve<4, NX>(P, key + 1, false, p0, dred, rec, C, it, tab, rt, alpha, rho); break;
      }
    }
  }
}

// psi_red[c] = q_c + N t_c over the reduced rows, for every own column c (the
// second half of Psi-comp).  16 consecutive rows per half warp (conflict-free
// with an odd number of 16-byte units per row); the two halves of a warp cover
// the two halves of the columns of the same rows.
template <int NX, int GT>
__device__ __forceinline__ void apply_n(const float *Nb, const float *tv, const float *q_p, int dred, int dred_pad,
                                        int kpad, int ldr, float *out, int gt) {
  constexpr int kWarps = GT / 32;
  const int ncg = kpad >> 2;
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
              const float4 t4 = *reinterpret_cast<const float4 *>(tv + c * kpad + 4 * (cg0 + u));
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
      for (int c = 0; c < NX; ++c) out[c * ldr + red] = o[c] + q_p[c * dred_pad + red];
    }
  }
}

// Conv of one patch from the per-thread squared residual partials (Sec. II-A
// stopping rule, per subsystem): ||Phi - Psi||_F <= eps_p and
// rho ||Psi - Psi_prev||_F <= eps_d.  The sums of squares are FP32 (per
// thread, then tree order over the warp and over the group's warps: relative
// error ~1e-6) and squared residuals are compared (no square root on the
// path).  GB300 runs FP64 at a small fraction of the FP32 rate, and the
// dependent FP64 chain this combine used to be (conversions, shuffles, adds,
// products on every patch of every iteration) sat on the iteration's critical
// path while adding nothing to a threshold test on FP32 partials.
template <int GT>
__device__ __forceinline__ void finish_item(const Params &P, int idx, const Item &it, const float *extra, Group &G,
                                            float prim_f, float dual_f, int g, int gt, unsigned *lnc, int iter) {
  constexpr int kWarps = GT / 32;
  const float prim_w = warp_sum_f(prim_f);
  const float dual_w = warp_sum_f(dual_f);
  if ((gt & 31) == 0) {
    G.red[2 * (gt >> 5)] = prim_w;
    G.red[2 * (gt >> 5) + 1] = dual_w;
  }
  group_sync(g, GT);
  if (gt < 32) {
    // lane w < kWarps holds warp w's sums; tree over the lanes
    constexpr int kTree = kWarps <= 1 ? 1 : kWarps <= 2 ? 2 : kWarps <= 4 ? 4 : 8;  // power of two >= kWarps
    float pp = gt < kWarps ? G.red[2 * gt] : 0.f;
    float dd = gt < kWarps ? G.red[2 * gt + 1] : 0.f;
#pragma unroll
    for (int o = kTree / 2; o > 0; o >>= 1) {
      pp += __shfl_xor_sync(0xffffffffu, pp, o);
      dd += __shfl_xor_sync(0xffffffffu, dd, o);
    }
    if (gt != 0) return;
    const float rho = extra[0], epsp = extra[1], epsd = extra[2];
    const bool conv = pp <= epsp * epsp && rho * rho * dd <= epsd * epsd;
    const float rj = sqrtf(pp);
    const float sj = rho * sqrtf(dd);
    P.item_r[idx] = rj;
    P.item_s[idx] = sj;
    if (!(isfinite(rj) && isfinite(sj))) set_error(P.err, DLMPC_ERR_NONFINITE, blockIdx.x, iter, it.sub);
    if (!conv) atomicAdd(lnc + it.lslot, 1u);
  }
}

// Psi-comp, Lambda-comp and the residuals of one patch, from the stored Psi
// and Lambda (the first iteration of a launch, and every iteration when Phi
// is exported).  With `cp` set it also starts the compact iterate: t0 = t,
// Y = 0, R = sum_c x_c Psi_c over the reduced rows.
template <int NX, int GT>
__device__ void project_item(const Params &P, int idx, const Item &it, const float *tab, const float *extra, Group &G,
                             const float *alpha, float *arena, float *Gnext, int g, int gt, unsigned *lnc, int iter,
                             float *cp, bool tr) {
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
      const float a = alpha[red];
#pragma unroll
      for (int c = 0; c < NX; ++c) G.vred[c * ldr + red] = psi_p[c * dcol + f] + a * xj[c];
    }
  }
  // N: resident in the arena, otherwise read from global memory (L2); the
  // generic 16-byte loads below serve both.
  const float *Nb = it.n_sm >= 0 ? arena + it.n_sm : P.Nmat + it.n_off;
  group_sync(g, GT);

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
        for (int rb = 2 * w + hw; rb < dred; rb += 4 * kStep) {
          float4 n4[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int red = rb + u * kStep;
            n4[u] = red < dred ? *reinterpret_cast<const float4 *>(nb + red * kpad) : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int red = rb + u * kStep;
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
  const int cpl = (dcol + 3) & ~3;  // compact iterate: lhat, R, Y, t0
  for (int e = gt; e < NX * kpad; e += GT) {
    const int c = e / kpad, a = e - c * kpad;
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += G.part[(w * NX + c) * kpad + a];
    s = (a < k) ? s : 0.f;  // padded columns of N are zero; keep t finite there
    G.t[c * kpad + a] = s;
    if (cp) {
      cp[cpl + it.dred_pad + kpad + e] = s;
      if (c == 0) cp[cpl + it.dred_pad + a] = 0.f;
    }
  }
  group_sync(g, GT);
  if (tr) trace_point(P, iter, 7);

  // pass 2: psi_red = q + N t
  apply_n<NX, GT>(Nb, G.t, q_p, dred, it.dred_pad, kpad, ldr, G.psired, gt);
  group_sync(g, GT);
  if (tr) trace_point(P, iter, 6);

  // slot-0 states pinned to e_c; Lambda-comp; residuals; new exchange sums
  float prim_f = 0.f, dual_f = 0.f;  // FP32 partials per thread, then per warp and per group
  for (int f = gt, mpos = mpos0, r = r0; f < dcol; f += GT, mpos += dm, r += dr) {
    if (r >= r_sub) { r -= r_sub; ++mpos; }
    const int red = mpos * rs_red + r - NX;
    const float a = alpha[r >= NX ? red : dred + mpos * NX + r];
    float gsum = 0.f, rsum = 0.f;
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
      rsum = fmaf(ps, xj[c], rsum);
    }
    if (cp && r >= NX) cp[cpl + red] = rsum;
    const int gi = reinterpret_cast<const int *>(tab + mpos * MT)[3] + r;
    Gnext[gi] = send(P, iter, it.sub, P.members + it.mem_off + mpos, gi, gsum);
  }
  finish_item<GT>(P, idx, it, extra, G, prim_f, dual_f, g, gt, lnc, iter);
}

// o = N y by rows of N (row-major, kpad floats per row, an odd number of
// 16-byte units so the rows of a warp hit distinct bank groups) with the sums
// of the flat pass over N^T, bit for bit: that pass gives partial q (q < QS)
// the terms a = q (mod QS) in increasing a, fused multiply-adds from zero,
// and the partials are added to zero in order q = 0, 1, ...; here partial q
// takes the same terms in the same order (QS in {1, 2, 4} divides the four
// entries of a 16-byte unit), and o[red] is that ordered sum.  The padded
// entries of N and y are zeros and add exact zeros.  Used by the 72- and
// 80-register tiers only (ROWS): at 64 registers its live values would add
// spills to the whole loop.
__device__ __forceinline__ void rows_pass(const float *Nb, int dred, int kpad, const float *y, float *o_out, int QS,
                                          int gt, int GT) {
  for (int red = gt; red < dred; red += GT) {
    const float *nr = Nb + red * kpad;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int c = 0; c < kpad; c += 4) {
      const float4 n4 = *reinterpret_cast<const float4 *>(nr + c);
      const float4 y4 = *reinterpret_cast<const float4 *>(y + c);
      if (QS == 1) {
        a0 = fmaf(n4.x, y4.x, a0);
        a0 = fmaf(n4.y, y4.y, a0);
        a0 = fmaf(n4.z, y4.z, a0);
        a0 = fmaf(n4.w, y4.w, a0);
      } else if (QS == 2) {
        a0 = fmaf(n4.x, y4.x, a0);
        a1 = fmaf(n4.y, y4.y, a1);
        a0 = fmaf(n4.z, y4.z, a0);
        a1 = fmaf(n4.w, y4.w, a1);
      } else {
        a0 = fmaf(n4.x, y4.x, a0);
        a1 = fmaf(n4.y, y4.y, a1);
        a2 = fmaf(n4.z, y4.z, a2);
        a3 = fmaf(n4.w, y4.w, a3);
      }
    }
    float o = 0.f;
    o += a0;
    if (QS >= 2) o += a1;
    if (QS == 4) {
      o += a2;
      o += a3;
    }
    o_out[red] = o;
  }
}

// Psi-comp, Lambda-comp and Conv of one patch on the compact iterate (every
// iteration after the first of a launch).  Once Psi_old = q + N t is a
// projected iterate, N^T q = 0 and N^T N = I turn the projection of
// v_c = Psi_old,c + alpha x_c into q_c + N (t_c + x_c y) with the single
// vector y = N^T alpha (reduced rows).  With o = N y and s = ||x_j||^2:
//   Psi_new,c - Psi_old,c = x_c o                (reduced rows; slot-0 rows fixed)
//   Lambda_new,c = x_c lhat,  lhat = alpha - o   (reduced rows), alpha (slot-0 rows)
//   R_new = R_old + s o,  R = sum_c x_c Psi_c over the reduced rows
//   exchange sum of a row: sum_c x_c (Psi_new - Lambda_new)_c = R_new - s lhat
//   ||Psi_new - Psi_old||^2 = s ||o||^2,  ||Lambda_new - Lambda_old||^2 = s ||lhat - lhat_old||^2
// so an iteration reads N and N^T once each with one right-hand side and
// touches neither Psi nor Lambda; Psi = q + N (t0 + x_c Y), Y = sum of the y,
// and Lambda = x_c lhat are formed once at the end of the launch.  `first`:
// Lambda_old is the stored Lambda of the first iteration, not yet of the form
// x_c lhat.
//
// Both passes read their matrix flat (flat_pass): thread (q, g) owns the
// 16-byte column group g of every QS-th row starting at row q, so a warp reads
// consecutive 16-byte units, and the QS partial sums per output are added
// afterwards.
template <int NX, int GT, bool ROWS>
__device__ void project_compact(const Params &P, int idx, const Item &it, const float *tab, const float *rt,
                                const float *extra, Group &G, const float *alpha, float *arena, float *Gnext, int g,
                                int gt, unsigned *lnc, int iter, bool first, bool tr) {
  const int MT = member_record(NX, P.nu);
  const int r_sub = it.r_sub;
  const int dcol = r_sub * it.n_mem;
  const int rs_red = r_sub - NX;
  const int dred = it.dred, dpad = it.dred_pad;
  const int k = it.k, kpad = it.kpad;
  float *cp = it.cp_sm >= 0 ? arena + it.cp_sm : P.cpst + it.cp_off;
  float *lhat = cp;
  float *Rv = cp + ((dcol + 3) & ~3);
  float *Y = Rv + dpad;
  const float *lam_p = it.st_sm >= 0 ? arena + it.st_sm + NX * dcol : P.Lam + it.st_off;
  const float *Nb = it.n_sm >= 0 ? arena + it.n_sm : P.Nmat + it.n_off;
  const float *NTb = P.Nmat + it.n_off + dpad * kpad;  // N^T (k x dred_pad) follows N in global memory
  float xj[NX];
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < NX; ++c) {
    xj[c] = tab[it.self_pos * MT + 4 + c];
    s = fmaf(xj[c], xj[c], s);
  }

  // pass 1: y = N^T alpha_red; Y += y
  flat_pass<8>(Nb, dred, kpad, alpha, G.part, gt, GT);
  group_sync(g, GT);
  {
    const int ncg = kpad >> 2;
    const int QS = GT >= ncg ? small_div(GT, ncg) : 1;
    for (int a = gt; a < kpad; a += GT) {
      float y = 0.f;
      if (a < k)
        for (int q = 0; q < QS; ++q) y += G.part[q * kpad + a];
      G.t[a] = y;
      Y[a] += y;
    }
  }
  group_sync(g, GT);
  if (tr) trace_point(P, iter, 7);

  // pass 2: o = N y.  A patch whose N is resident takes it by rows from
  // shared memory (no L2 traffic); the others read N^T from L2 flat.
  const int nrg = dpad >> 2;
  const int QS2 = GT >= nrg ? small_div(GT, nrg) : 1;
  const bool by_rows = ROWS && it.n_sm >= 0 && (QS2 == 1 || QS2 == 2 || QS2 == 4);
  if (by_rows) rows_pass(Nb, dred, kpad, G.t, G.part, QS2, gt, GT);
  else flat_pass<8>(NTb, k, dpad, G.t, G.part, gt, GT);
  group_sync(g, GT);
  if (tr) trace_point(P, iter, 6);

  // Lambda-comp, residuals and exchange sums of the reduced rows
  float prim_f = 0.f, dual_f = 0.f;
  {
    const int QS = by_rows ? 1 : QS2;
    for (int red = gt; red < dred; red += GT) {
      float o = 0.f;
      for (int q = 0; q < QS; ++q) o += G.part[q * dpad + red];
      const float lh = alpha[red] - o;
      if (first) {
        const int mpos = red / rs_red, f = red + (mpos + 1) * NX;
#pragma unroll
        for (int c = 0; c < NX; ++c) {
          const float dp = xj[c] * lh - lam_p[c * dcol + f];
          prim_f = fmaf(dp, dp, prim_f);
        }
      } else {
        const float dp = lh - lhat[red];
        prim_f = fmaf(s * dp, dp, prim_f);
      }
      dual_f = fmaf(s * o, o, dual_f);
      const float rn = fmaf(s, o, Rv[red]);
      Rv[red] = rn;
      lhat[red] = lh;
      const int mpos = small_div(red, rs_red);
      const int gi = P.rows_cached ? reinterpret_cast<const int *>(rt + red * kRowRecord)[2]
                                   : reinterpret_cast<const int *>(tab + mpos * MT)[3] + red - mpos * rs_red + NX;
      Gnext[gi] = send(P, iter, it.sub, P.members + it.mem_off + mpos, gi, fmaf(-s, lh, rn));
    }
  }
  // slot-0 rows: Psi fixed (e_c on the own member), lhat = alpha
  for (int p = dred + gt; p < dcol; p += GT) {
    const float a = alpha[p];
    if (first) {
      const int mpos = (p - dred) / NX, f = mpos * r_sub + (p - dred - mpos * NX);
#pragma unroll
      for (int c = 0; c < NX; ++c) {
        const float dp = xj[c] * a - lam_p[c * dcol + f];
        prim_f = fmaf(dp, dp, prim_f);
      }
    } else {
      const float dp = a - lhat[p];
      prim_f = fmaf(s * dp, dp, prim_f);
    }
    lhat[p] = a;
    const RowRec rr = get_row<NX>(P, it, tab, rt, p);
    const int aux = rr.aux;
    float own = 0.f;
#pragma unroll
    for (int c = 0; c < NX; ++c)
      if (aux == c) own = xj[c];
    const int gi = rr.wr;
    Gnext[gi] = send(P, iter, it.sub, P.members + it.mem_off + small_div(p - dred, NX), gi, fmaf(-s, a, own));
  }
  finish_item<GT>(P, idx, it, extra, G, prim_f, dual_f, g, gt, lnc, iter);
}

// End of a launch whose last iteration ran on the compact iterate: Psi_c =
// q_c + N (t0_c + x_c Y) (slot-0 rows e_c) and Lambda_c = x_c lhat, written
// to the global state.
template <int NX, int GT>
__device__ void expand_compact(const Params &P, const Item &it, Group &G, float *arena, int g, int gt) {
  const int r_sub = it.r_sub;
  const int dcol = r_sub * it.n_mem;
  const int rs_red = r_sub - NX;
  const int dred = it.dred, k = it.k, kpad = it.kpad;
  const int ldr = P.max_dred_pad;
  const float *cp = it.cp_sm >= 0 ? arena + it.cp_sm : P.cpst + it.cp_off;
  const float *lhat = cp;
  const float *Y = cp + ((dcol + 3) & ~3) + it.dred_pad;
  const float *t0 = Y + kpad;
  const float *Nb = it.n_sm >= 0 ? arena + it.n_sm : P.Nmat + it.n_off;
  const float *q_p = it.q_sm >= 0 ? arena + it.q_sm : P.qvec + it.q_off;
  float xj[NX];
#pragma unroll
  for (int c = 0; c < NX; ++c) xj[c] = P.x[(int64_t)it.sub * NX + c];
  for (int e = gt; e < NX * kpad; e += GT) {
    const int c = e / kpad, a = e - c * kpad;
    float xc = 0.f;
#pragma unroll
    for (int cc = 0; cc < NX; ++cc)
      if (cc == c) xc = xj[cc];
    G.t[e] = (a < k) ? fmaf(xc, Y[a], t0[e]) : 0.f;
  }
  group_sync(g, GT);
  apply_n<NX, GT>(Nb, G.t, q_p, dred, it.dred_pad, kpad, ldr, G.psired, gt);
  group_sync(g, GT);
  for (int e = gt; e < NX * dcol; e += GT) {
    const int c = e / dcol, f = e - c * dcol;
    const int mpos = f / r_sub, r = f - mpos * r_sub;
    const int red = mpos * rs_red + r - NX;
    float xc = 0.f;
#pragma unroll
    for (int cc = 0; cc < NX; ++cc)
      if (cc == c) xc = xj[cc];
    const float ps = (r < NX) ? ((mpos == it.self_pos && r == c) ? 1.f : 0.f) : G.psired[c * ldr + red];
    P.Psi[it.st_off + e] = ps;
    P.Lam[it.st_off + e] = xc * lhat[r >= NX ? red : dred + mpos * NX + r];
  }
  group_sync(g, GT);
}

__device__ __forceinline__ void red_add_release_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// CTA-wide bounded barrier on the rotating 64-bit counter of barrier number e.
// Returns false on timeout or when any CTA has recorded an error; `total` is
// the number of not-converged patches summed over the grid.
__device__ __forceinline__ bool sweep_barrier(const Params &P, unsigned e, unsigned my_nc, unsigned long long *prev_hi,
                                              unsigned &total, int iter, bool synced = false) {
  __shared__ int ok_sh;
  __shared__ unsigned total_sh;
  if (!synced) __syncthreads();  // the CTA's writes before the arrival (the caller may have synchronised)
  if (threadIdx.x == 0) {
    unsigned long long *ctr = P.bar + (e % 3);
    red_add_release_u64(ctr, 1ull | ((unsigned long long)my_nc << 32));
    const unsigned target = (e / 3 + 1) * gridDim.x;
    const unsigned long long t0 = global_ns();
    int ok = 1;
    unsigned long long v = 0;
    for (unsigned spins = 0;; ++spins) {
      v = ld_acquire_u64(ctr);  // (measured: cheaper than relaxed polls plus one fence)
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

// BLK: the Phi-step takes full cost blocks (phi_slots); a separate
// instantiation keeps that solver out of the diagonal kernel's registers.
// MAXT: the most threads a CTA of this instantiation may have, which sets its
// register budget (65536 / MAXT per thread): 1024 gives 64 registers, 896
// gives 72 and 768 gives 80, enough for the loop to run without spills.
template <int NX, int GT, bool BLK, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) sweep_kernel(Params P) {
  extern __shared__ __align__(16) float sm[];
  const int tid = threadIdx.x;
  const int g = tid / GT, gt = tid - g * GT;
  const int b = blockIdx.x;
  const GroupLayout L =
      group_layout(NX, P.nu, GT, P.wave, P.max_dcol, P.max_dred_pad, P.max_kpad, P.max_nmem, P.rows_cached != 0);
  float *gbase = sm + g * P.grp_floats;
  Group G;
  G.alpha = gbase + L.alpha;
  G.vred = gbase + L.vred;
  G.psired = gbase + L.psired;
  G.t = gbase + L.t;
  G.part = gbase + L.part;
  G.red = gbase + L.red;
  G.mtab = gbase + L.mtab;
  G.rtab = gbase + L.rtab;
  G.icache = gbase + L.icache;
  G.mbar = reinterpret_cast<uint64_t *>(gbase + L.mbar);
  G.phase = 0;
  float *cta = sm + P.ng * P.grp_floats;
  unsigned long long *prev_hi = reinterpret_cast<unsigned long long *>(cta);  // [3] (+1 pad)
  unsigned *lnc = reinterpret_cast<unsigned *>(cta + 8);                      // [max_local_inst]
  int *lact = reinterpret_cast<int *>(cta + 8 + P.max_local_inst);            // [max_local_inst]
  int *lcnt = reinterpret_cast<int *>(cta + 8 + 2 * P.max_local_inst);        // [max_local_inst] iterations run
  float *arena = cta + P.cta_floats;

  const int gi0 = P.grp_ptr[b * P.ng + g];
  const int gi1 = P.grp_ptr[b * P.ng + g + 1];
  const int li0 = P.cta_inst_ptr[b], nli = P.cta_inst_ptr[b + 1] - li0;
  const bool one_wave = gi1 - gi0 <= P.wave;  // member tables filled once per launch

  // the word after the mbarrier: 0, or 1 + the parity of a bulk copy whose
  // wait ran out (the group then issues no further copies)
  volatile int *cfail = reinterpret_cast<volatile int *>(G.mbar + 1);
  if (gt == 0) {
    mbar_init(G.mbar, 1);
    *cfail = 0;
  }
  if (tid < 3) prev_hi[tid] = 0ull;
  for (int t = tid; t < nli; t += blockDim.x) lcnt[t] = 0;
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
    // start: zeros, or the state left by the previous step (with
    // DLMPC_WARM_CONVERGED only where that step met Conv)
    const bool warm_i = P.warm == DLMPC_WARM_PREVIOUS || (P.warm == DLMPC_WARM_CONVERGED && P.conv_prev[it.inst] != 0);
    for (int e = gt; e < NX * dcol; e += GT) {
      const float ps = warm_i ? psi_g[e] : 0.f;
      const float lm = warm_i ? lam_g[e] : 0.f;
      psi_p[e] = ps;
      lam_p[e] = lm;
    }
    if (it.q_sm >= 0)
      for (int e = gt; e < NX * it.dred_pad; e += GT) arena[it.q_sm + e] = P.qvec[it.q_off + e];
    if (it.n_sm >= 0) {
      if (*cfail == 0) {
        if (gt == 0) tma_load_1d(arena + it.n_sm, P.Nmat + it.n_off, (unsigned)it.dred_pad * it.kpad * 4u, G.mbar);
        if (!mbar_wait(G.mbar, G.phase & 1u, P.timeout_ns)) {
          ok = false;
          *cfail = 1 + (int)(G.phase & 1u);
        }
        ++G.phase;
      } else {
        ok = false;  // an earlier copy of this group timed out: no loop will run
      }
    }
    group_sync(g, GT);
    if constexpr (BLK) {
      // explicit solution of the own subsystem's slot QPs for this x(tau)
      const float s_own = __ldcg(P.S + it.sub);
      if (P.expl && s_own > 0.f) {
        const float cd = P.rho_i[it.inst] * (1.f / s_own);
        const int nrx = P.rg_cnt[2 * it.sub], nr = nrx + P.rg_cnt[2 * it.sub + 1];
        for (int e = gt; e < nr; e += GT) {
          if (e < nrx) {
            build_region<NX>(P, it.sub, 0, e, cd);
          } else {
            switch (P.nu) {
              case 1: build_region<1>(P, it.sub, 1, e - nrx, cd); break;
              case 2: build_region<2>(P, it.sub, 1, e - nrx, cd); break;
              case 3: build_region<3>(P, it.sub, 1, e - nrx, cd); break;
              default: build_region<4>(P, it.sub, 1, e - nrx, cd); break;
            }
          }
        }
      }
    }
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
    fill_wave<NX>(P, P.grp_items + gi0, gi1 - gi0, G.icache, G.mtab, G.rtab, g, gt, GT);
    group_sync(g, GT);
  }

  // ---- ADMM iterations (Alg. 2)
  const int n_it = P.fixed_iters > 0 ? P.fixed_iters : P.max_iter;
  const bool multi = P.n_inst > 1;
  const bool compact = P.compact != 0 && P.Phi == nullptr;
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
        active = __ldcg(P.notconv + prev * P.n_inst + P.cta_inst[li0 + t]) > 0u;
      lact[t] = active;
      lcnt[t] += active;
    }
    __syncthreads();
    trace_point(P, iter, 0);
    const float *Gcur = (iter & 1) ? P.G1 : P.G0;
    float *Gnext = (iter & 1) ? P.G0 : P.G1;
    for (int w0 = gi0; w0 < gi1; w0 += P.wave) {
      const int wn = min(P.wave, gi1 - w0);
      if (!one_wave) {
        group_sync(g, GT);  // the previous wave is done with the cache
        fill_wave<NX>(P, P.grp_items + w0, wn, G.icache, G.mtab, G.rtab, g, gt, GT);
        group_sync(g, GT);
      }
      for (int wi = 0; wi < wn; ++wi) {
        const Item &it = cached_item(G.icache, wi);
        if (!lact[it.lslot]) continue;
        // the record source is chosen once per patch, not per row
        if (P.rows_cached)
          phi_rows<NX, GT, BLK, true>(P, it, G.mtab + wi * P.max_nmem * MT, G.rtab + wi * P.max_dcol * kRowRecord,
                                      Gcur, G.alpha + wi * P.max_dcol, gt);
        else
          phi_rows<NX, GT, BLK, false>(P, it, G.mtab + wi * P.max_nmem * MT, nullptr, Gcur, G.alpha + wi * P.max_dcol,
                                       gt);
      }
      if constexpr (BLK) {
        group_sync(g, GT);  // every row's w is in alpha
        for (int wi = 0; wi < wn; ++wi) {
          const Item &it = cached_item(G.icache, wi);
          if (!lact[it.lslot]) continue;
          phi_slots<NX>(P, it, G.mtab + wi * P.max_nmem * MT, G.rtab + wi * P.max_dcol * kRowRecord,
                        G.alpha + wi * P.max_dcol, cached_extra(G.icache, wi)[0], gt, GT);
        }
      }
      group_sync(g, GT);
      if (w0 == gi0) trace_point(P, iter, 1);
      for (int wi = 0; wi < wn; ++wi) {
        const Item &it = cached_item(G.icache, wi);
        if (!lact[it.lslot]) continue;
        const float *ex = cached_extra(G.icache, wi);
        const int idx = reinterpret_cast<const int *>(ex)[3];
        const bool tr = w0 == gi0 && wi == 0;
        if (compact && iter > 0)
          project_compact<NX, GT, (MAXT <= 896)>(P, idx, it, G.mtab + wi * P.max_nmem * MT,
                                  G.rtab + wi * P.max_dcol * kRowRecord, ex, G, G.alpha + wi * P.max_dcol, arena,
                                  Gnext, g, gt, lnc, iter, iter == 1, tr);
        else
          project_item<NX, GT>(P, idx, it, G.mtab + wi * P.max_nmem * MT, ex, G, G.alpha + wi * P.max_dcol, arena,
                               Gnext, g, gt, lnc, iter,
                               compact ? (it.cp_sm >= 0 ? arena + it.cp_sm : P.cpst + it.cp_off) : nullptr, tr);
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
    ok = sweep_barrier(P, e_bar++, my_nc, prev_hi, total, iter, true);
    if (!ok) break;
    trace_point(P, iter, 5);
    if (b == 0) {
      if (multi) {
        for (int e = tid; e < P.n_inst; e += blockDim.x)
          if (P.inst_iters[e] == 0 && __ldcg(P.notconv + slot * P.n_inst + e) == 0u) P.inst_iters[e] = iter + 1;
      } else if (tid == 0 && total == 0u && P.inst_iters[0] == 0) {
        P.inst_iters[0] = iter + 1;
      }
    }
    if (P.fixed_iters <= 0 && total == 0u) { ++iter; break; }
  }
  if (b == 0 && tid == 0) P.err[4] = iter;
  // every CTA is past its prologue (the grid barriers): record which
  // instances met Conv, the next DLMPC_WARM_CONVERGED step reads it (each
  // thread of CTA 0 reads the counts it wrote itself)
  if (b == 0)
    for (int e = tid; e < P.n_inst; e += blockDim.x) P.conv_prev[e] = (ok && P.inst_iters[e] > 0) ? 1 : 0;

  // ---- epilogue: final Psi/Lambda (from the compact iterate, or the resident
  // state written back), dynamics
  __syncthreads();
  for (int ii = gi0; ii < gi1; ++ii) {
    const Item &it = P.items[P.grp_items[ii]];
    if (compact && lcnt[it.lslot] >= 2) {
      expand_compact<NX, GT>(P, it, G, arena, g, gt);
      continue;
    }
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
  if (*cfail != 0) {
    // a timed-out bulk copy may still be landing in the arena: wait for it
    // once more (bounded) before the CTA gives up its shared memory, and
    // invalidate the barrier only if it has completed
    const bool done = mbar_wait(G.mbar, (unsigned)(*cfail - 1), P.timeout_ns);
    if (done && gt == 0) mbar_inval(G.mbar);
  } else if (gt == 0) {
    mbar_inval(G.mbar);
  }
}

}  // namespace dlmpc
