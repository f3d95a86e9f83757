// Learned warm start for the ADMM (the paper names a better initial point as
// future work, Sec. V): a three-layer MLP
//     h1 = GELU(x W1 + b1), h2 = GELU(h1 W2 + b2), y = h2 W3 + b3
// with BF16 operands and FP32 accumulation on the tensor cores
// (mma.sync m16n8k16), FP32 master weights and AdamW.  The GEMMs here are
// small (n x d_in x 256, n x 256 x 256, n x 256 x d_out); one generic tiled
// kernel serves the forward (bias and GELU fused into its epilogue) and both
// backward products.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dlmpc.h"

namespace {

constexpr int kTile = 64;   // CTA tile (M and N)
constexpr int kKc = 64;     // K per staged chunk (four m16n8k16 steps)
constexpr int kLd = 72;     // padded row (bf16) of a shared tile: conflict-free 32-bit fragment loads
constexpr int kPairs = kTile * kKc / 2 / 128;  // bf16 pairs per thread per operand chunk

__device__ __forceinline__ uint32_t pack2(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float gelu(float x);

// One operand chunk (kTile rows of the M or N side x kKc of K) as kPairs
// pairs of bf16 per thread, read along the source's contiguous dimension.  kcont: the
// source is contiguous along K (src[r * ld + k]); otherwise along the row
// index (src[k * ld + r]).  Out-of-range elements read as zero.
struct Chunk {
  uint32_t v[kPairs];
};

__device__ __forceinline__ uint32_t pair_bits(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void load_chunk(Chunk &c, const __nv_bfloat16 *src, int ld, bool kcont, bool pairs,
                                           int r0, int rmax, int k0, int kmax, int tid) {
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
#pragma unroll
  for (int i = 0; i < kPairs; ++i) {
    const int e = tid + 128 * i;
    int r, k, r2, k2;
    if (kcont) {
      r = r0 + (e >> 5);
      k = k0 + 2 * (e & 31);
      r2 = r;
      k2 = k + 1;
    } else {
      k = k0 + (e >> 5);
      r = r0 + 2 * (e & 31);
      k2 = k;
      r2 = r + 1;
    }
    const bool in1 = r < rmax && k < kmax, in2 = r2 < rmax && k2 < kmax;
    const int64_t o1 = kcont ? (int64_t)r * ld + k : (int64_t)k * ld + r;
    if (pairs && in1 && in2) {
      c.v[i] = *reinterpret_cast<const uint32_t *>(src + o1);
    } else {
      const __nv_bfloat16 x1 = in1 ? src[o1] : zero;
      const __nv_bfloat16 x2 = in2 ? src[o1 + 1] : zero;
      c.v[i] = pair_bits(x1, x2);
    }
  }
}

// Writes a chunk into the shared tile T[row][k] (row = M or N index).
__device__ __forceinline__ void store_chunk(const Chunk &c, __nv_bfloat16 (*T)[kLd], bool kcont, int tid) {
#pragma unroll
  for (int i = 0; i < kPairs; ++i) {
    const int e = tid + 128 * i;
    if (kcont) {
      *reinterpret_cast<uint32_t *>(&T[e >> 5][2 * (e & 31)]) = c.v[i];
    } else {
      const int kk = e >> 5, rr = 2 * (e & 31);
      T[rr][kk] = __ushort_as_bfloat16((unsigned short)(c.v[i] & 0xffffu));
      T[rr + 1][kk] = __ushort_as_bfloat16((unsigned short)(c.v[i] >> 16));
    }
  }
}

// C[M x N] (+)= op(A)[M x K] op(B)[K x N]; op(A) = A (A[m*lda+k]) or A^T
// (A[k*lda+m]); op(B) = B (B[k*ldb+n]) or B^T (B[n*ldb+k]).  BF16 inputs,
// FP32 accumulate.  128 threads, 4 warps of 32x32; K staged in chunks of 64
// through shared memory, the next chunk loaded into registers while the
// current one is multiplied.  Epilogue: epi = 0 stores (or adds) C;
// epi = 1 adds bias[n], stores C (pre-activation) and act = BF16(GELU(C));
// epi = 2 adds bias[n], stores C and out = C * scale[n] + shift[n] (or C
// when scale is null) when out is given.
struct Epilogue {
  int epi;
  const float *bias;
  __nv_bfloat16 *act;
  float *out;
  const float *scale, *shift;
};

__global__ void __launch_bounds__(128) gemm_bf16_kernel(int M, int N, int K, const __nv_bfloat16 *A, int lda, int ta,
                                                        const __nv_bfloat16 *B, int ldb, int tb, float *C, int ldc,
                                                        int accumulate, Epilogue ep) {
  __shared__ __align__(16) __nv_bfloat16 As[kTile][kLd];  // [m][k]
  __shared__ __align__(16) __nv_bfloat16 Bs[kTile][kLd];  // [n][k]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int bm = blockIdx.y * kTile, bn = blockIdx.x * kTile;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const bool a_k = ta == 0, b_k = tb != 0;  // operand contiguous along K
  const bool a_pairs = (lda % 2) == 0 && (reinterpret_cast<uintptr_t>(A) & 3) == 0;
  const bool b_pairs = (ldb % 2) == 0 && (reinterpret_cast<uintptr_t>(B) & 3) == 0;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
  Chunk ca, cb;
  load_chunk(ca, A, lda, a_k, a_pairs, bm, M, 0, K, tid);
  load_chunk(cb, B, ldb, b_k, b_pairs, bn, N, 0, K, tid);
  for (int k0 = 0; k0 < K; k0 += kKc) {
    store_chunk(ca, As, a_k, tid);
    store_chunk(cb, Bs, b_k, tid);
    __syncthreads();
    if (k0 + kKc < K) {
      load_chunk(ca, A, lda, a_k, a_pairs, bm, M, k0 + kKc, K, tid);
      load_chunk(cb, B, ldb, b_k, b_pairs, bn, N, k0 + kKc, K, tid);
    }
#pragma unroll
    for (int ks = 0; ks < kKc; ks += 16) {
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int m0 = wm + 16 * i;
        const uint32_t a0 = pack2(&As[m0 + g][ks + 2 * t]);
        const uint32_t a1 = pack2(&As[m0 + g + 8][ks + 2 * t]);
        const uint32_t a2 = pack2(&As[m0 + g][ks + 2 * t + 8]);
        const uint32_t a3 = pack2(&As[m0 + g + 8][ks + 2 * t + 8]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int n0 = wn + 8 * j;
          const uint32_t b0 = pack2(&Bs[n0 + g][ks + 2 * t]);
          const uint32_t b1 = pack2(&Bs[n0 + g][ks + 2 * t + 8]);
          mma_bf16(acc[i][j], a0, a1, a2, a3, b0, b1);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int m = bm + wm + 16 * i + g + ((e >> 1) << 3);
        const int n = bn + wn + 8 * j + 2 * t + (e & 1);
        if (m < M && n < N) {
          const int64_t o = (int64_t)m * ldc + n;
          float v = acc[i][j][e];
          if (ep.epi == 0) {
            C[o] = accumulate ? C[o] + v : v;
          } else {
            v += ep.bias[n];
            C[o] = v;
            if (ep.epi == 1) ep.act[o] = __float2bfloat16(gelu(v));
            else if (ep.out) ep.out[o] = ep.scale ? v * ep.scale[n] + ep.shift[n] : v;
          }
        }
      }
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__global__ void to_bf16_kernel(const float *in, __nv_bfloat16 *out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16(in[i]);
}

// dy = 2 (y - t) / (n d), loss partial sums of (y - t)^2 (FP64 atomics).
__global__ void mse_grad_kernel(const float *y, const float *tgt, int64_t total, float inv, __nv_bfloat16 *dy_bf,
                                float *dy, double *loss) {
  double local = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const float r = y[i] - tgt[i];
    local += (double)r * r;
    const float gval = 2.f * r * inv;
    dy[i] = gval;
    dy_bf[i] = __float2bfloat16(gval);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, local);
}

// dh = da * GELU'(pre) (FP32 and BF16 copies).
__global__ void gelu_back_kernel(const float *da, const float *pre, int64_t total, float *dh, __nv_bfloat16 *dh_bf) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = da[i] * gelu_grad(pre[i]);
    dh[i] = v;
    dh_bf[i] = __float2bfloat16(v);
  }
}

// db[c] = sum_rows d[r][c]
__global__ void col_sum_kernel(const float *d, int n, int cols, float *db) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < n; ++r) s += d[(int64_t)r * cols + c];
  db[c] = s;
}

// AdamW on FP32 masters; refreshes the BF16 copy of the weights.
__global__ void adamw_kernel(float *w, const float *grad, float *m, float *v, __nv_bfloat16 *w_bf, int64_t n,
                             float lr, float b1, float b2, float eps, float wd, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gr = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gr;
    const float vi = b2 * v[i] + (1.f - b2) * gr * gr;
    m[i] = mi;
    v[i] = vi;
    float wi = w[i] * (1.f - lr * wd);
    wi -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (w_bf) w_bf[i] = __float2bfloat16(wi);
  }
}

int blocks_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

}  // namespace

// ---------------------------------------------------------------------------
// the MLP object
// ---------------------------------------------------------------------------

struct dlmpc_mlp {
  int d_in = 0, hid = 0, d_out = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  int64_t n_params = 0;
  // parameter layout (FP32 masters, one contiguous block):
  // W1 [d_in x hid], b1 [hid], W2 [hid x hid], b2 [hid], W3 [hid x d_out], b3 [d_out]
  int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
  float *w = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *w_bf = nullptr;  // BF16 copies of every parameter (biases unused)
  float *scale = nullptr, *shift = nullptr;  // output de-normalisation [d_out]
  int64_t step = 0;
  // activations for a batch of up to cap rows
  int cap = 0;
  __nv_bfloat16 *x_bf = nullptr, *h1_bf = nullptr, *h2_bf = nullptr, *dy_bf = nullptr, *dh2_bf = nullptr,
                *dh1_bf = nullptr;
  float *h1 = nullptr, *h2 = nullptr, *y = nullptr, *dy = nullptr, *da2 = nullptr, *dh2 = nullptr, *da1 = nullptr,
        *dh1 = nullptr;
  double *loss = nullptr;
  ~dlmpc_mlp() { release(); }
  void release_batch() {
    void *ps[] = {x_bf, h1_bf, h2_bf, dy_bf, dh2_bf, dh1_bf, h1, h2, y, dy, da2, dh2, da1, dh1};
    for (void *p : ps)
      if (p) cudaFree(p);
    x_bf = h1_bf = h2_bf = dy_bf = dh2_bf = dh1_bf = nullptr;
    h1 = h2 = y = dy = da2 = dh2 = da1 = dh1 = nullptr;
    cap = 0;
  }
  void release() {
    release_batch();
    void *ps[] = {w, grad, m, v, w_bf, scale, shift, loss};
    for (void *p : ps)
      if (p) cudaFree(p);
    w = grad = m = v = scale = shift = nullptr;
    w_bf = nullptr;
    loss = nullptr;
  }
  int fail(int code, const std::string &msg) {
    err = msg;
    return code;
  }
};

#define MK(call, what)                                                       \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) return mlp->fail(DLMPC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
  } while (0)

namespace {

int ensure_batch(dlmpc_mlp *mlp, int n) {
  if (n <= mlp->cap) return 0;
  mlp->release_batch();
  const int64_t H = (int64_t)n * mlp->hid, O = (int64_t)n * mlp->d_out, I = (int64_t)n * mlp->d_in;
  MK(cudaMalloc(&mlp->x_bf, I * 2), "alloc");
  MK(cudaMalloc(&mlp->h1_bf, H * 2), "alloc");
  MK(cudaMalloc(&mlp->h2_bf, H * 2), "alloc");
  MK(cudaMalloc(&mlp->dy_bf, O * 2), "alloc");
  MK(cudaMalloc(&mlp->dh2_bf, H * 2), "alloc");
  MK(cudaMalloc(&mlp->dh1_bf, H * 2), "alloc");
  MK(cudaMalloc(&mlp->h1, H * 4), "alloc");
  MK(cudaMalloc(&mlp->h2, H * 4), "alloc");
  MK(cudaMalloc(&mlp->y, O * 4), "alloc");
  MK(cudaMalloc(&mlp->dy, O * 4), "alloc");
  MK(cudaMalloc(&mlp->da2, H * 4), "alloc");
  MK(cudaMalloc(&mlp->dh2, H * 4), "alloc");
  MK(cudaMalloc(&mlp->da1, H * 4), "alloc");
  MK(cudaMalloc(&mlp->dh1, H * 4), "alloc");
  mlp->cap = n;
  return 0;
}

int gemm(dlmpc_mlp *mlp, int M, int N, int K, const __nv_bfloat16 *A, int lda, int ta, const __nv_bfloat16 *B,
         int ldb, int tb, float *C, int ldc, int acc, Epilogue ep = Epilogue{0, nullptr, nullptr, nullptr, nullptr,
                                                                                nullptr}) {
  dim3 grid((N + kTile - 1) / kTile, (M + kTile - 1) / kTile);
  gemm_bf16_kernel<<<grid, 128, 0, mlp->stream>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, acc, ep);
  MK(cudaGetLastError(), "gemm_bf16_kernel");
  return 0;
}

// Forward pass; leaves pre-activations in h1/h2/y and BF16 activations.
// out (device, may be null) receives y de-normalised when `denorm`.
int forward(dlmpc_mlp *mlp, const float *x, int n, float *out, bool denorm) {
  int rc = ensure_batch(mlp, n);
  if (rc) return rc;
  cudaStream_t s = mlp->stream;
  const int I = mlp->d_in, H = mlp->hid, O = mlp->d_out;
  to_bf16_kernel<<<blocks_for((int64_t)n * I), 256, 0, s>>>(x, mlp->x_bf, (int64_t)n * I);
  // bias, GELU and the output de-normalisation run in the GEMM epilogues
  if ((rc = gemm(mlp, n, H, I, mlp->x_bf, I, 0, mlp->w_bf + mlp->oW1, H, 0, mlp->h1, H, 0,
                 Epilogue{1, mlp->w + mlp->ob1, mlp->h1_bf, nullptr, nullptr, nullptr})))
    return rc;
  if ((rc = gemm(mlp, n, H, H, mlp->h1_bf, H, 0, mlp->w_bf + mlp->oW2, H, 0, mlp->h2, H, 0,
                 Epilogue{1, mlp->w + mlp->ob2, mlp->h2_bf, nullptr, nullptr, nullptr})))
    return rc;
  if ((rc = gemm(mlp, n, O, H, mlp->h2_bf, H, 0, mlp->w_bf + mlp->oW3, O, 0, mlp->y, O, 0,
                 Epilogue{2, mlp->w + mlp->ob3, nullptr, out, denorm ? mlp->scale : nullptr, mlp->shift})))
    return rc;
  MK(cudaGetLastError(), "forward");
  return 0;
}

// Loss and gradients of the mean squared error against normalised targets.
int backward(dlmpc_mlp *mlp, const float *x, const float *tgt, int n) {
  int rc = forward(mlp, x, n, nullptr, false);
  if (rc) return rc;
  cudaStream_t s = mlp->stream;
  const int I = mlp->d_in, H = mlp->hid, O = mlp->d_out;
  const int64_t nO = (int64_t)n * O, nH = (int64_t)n * H;
  MK(cudaMemsetAsync(mlp->loss, 0, 8, s), "memset");
  mse_grad_kernel<<<blocks_for(nO), 256, 0, s>>>(mlp->y, tgt, nO, 1.f / (float)nO, mlp->dy_bf, mlp->dy, mlp->loss);
  // layer 3: dW3 = h2^T dy, db3 = sum dy, da2 = dy W3^T
  if ((rc = gemm(mlp, H, O, n, mlp->h2_bf, H, 1, mlp->dy_bf, O, 0, mlp->grad + mlp->oW3, O, 0))) return rc;
  col_sum_kernel<<<(O + 255) / 256, 256, 0, s>>>(mlp->dy, n, O, mlp->grad + mlp->ob3);
  if ((rc = gemm(mlp, n, H, O, mlp->dy_bf, O, 0, mlp->w_bf + mlp->oW3, O, 1, mlp->da2, H, 0))) return rc;
  gelu_back_kernel<<<blocks_for(nH), 256, 0, s>>>(mlp->da2, mlp->h2, nH, mlp->dh2, mlp->dh2_bf);
  // layer 2
  if ((rc = gemm(mlp, H, H, n, mlp->h1_bf, H, 1, mlp->dh2_bf, H, 0, mlp->grad + mlp->oW2, H, 0))) return rc;
  col_sum_kernel<<<(H + 255) / 256, 256, 0, s>>>(mlp->dh2, n, H, mlp->grad + mlp->ob2);
  if ((rc = gemm(mlp, n, H, H, mlp->dh2_bf, H, 0, mlp->w_bf + mlp->oW2, H, 1, mlp->da1, H, 0))) return rc;
  gelu_back_kernel<<<blocks_for(nH), 256, 0, s>>>(mlp->da1, mlp->h1, nH, mlp->dh1, mlp->dh1_bf);
  // layer 1
  if ((rc = gemm(mlp, I, H, n, mlp->x_bf, I, 1, mlp->dh1_bf, H, 0, mlp->grad + mlp->oW1, H, 0))) return rc;
  col_sum_kernel<<<(H + 255) / 256, 256, 0, s>>>(mlp->dh1, n, H, mlp->grad + mlp->ob1);
  MK(cudaGetLastError(), "backward");
  return 0;
}

}  // namespace

extern "C" int dlmpc_mlp_create(int32_t d_in, int32_t hidden, int32_t d_out, void *stream, dlmpc_mlp **out) {
  if (!out || d_in < 1 || hidden < 1 || d_out < 1) return DLMPC_ERR_ARG;
  *out = nullptr;
  auto *mlp = new (std::nothrow) dlmpc_mlp();
  if (!mlp) return DLMPC_ERR_NOMEM;
  mlp->d_in = d_in;
  mlp->hid = hidden;
  mlp->d_out = d_out;
  mlp->stream = static_cast<cudaStream_t>(stream);
  int64_t o = 0;
  mlp->oW1 = o; o += (int64_t)d_in * hidden;
  mlp->ob1 = o; o += hidden;
  mlp->oW2 = o; o += (int64_t)hidden * hidden;
  mlp->ob2 = o; o += hidden;
  mlp->oW3 = o; o += (int64_t)hidden * d_out;
  mlp->ob3 = o; o += d_out;
  mlp->n_params = o;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&mlp->w, o * 4);
  if (e == cudaSuccess) e = cudaMalloc(&mlp->grad, o * 4);
  if (e == cudaSuccess) e = cudaMalloc(&mlp->m, o * 4);
  if (e == cudaSuccess) e = cudaMalloc(&mlp->v, o * 4);
  if (e == cudaSuccess) e = cudaMalloc(&mlp->w_bf, o * 2);
  if (e == cudaSuccess) e = cudaMalloc(&mlp->scale, d_out * 4);
  if (e == cudaSuccess) e = cudaMalloc(&mlp->shift, d_out * 4);
  if (e == cudaSuccess) e = cudaMalloc(&mlp->loss, 8);
  if (e == cudaSuccess) e = cudaMemsetAsync(mlp->w, 0, o * 4, mlp->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(mlp->m, 0, o * 4, mlp->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(mlp->v, 0, o * 4, mlp->stream);
  if (e != cudaSuccess) {
    delete mlp;
    return e == cudaErrorMemoryAllocation ? DLMPC_ERR_NOMEM : DLMPC_ERR_CUDA;
  }
  std::vector<float> one(d_out, 1.f), zero(d_out, 0.f);
  cudaMemcpy(mlp->scale, one.data(), d_out * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(mlp->shift, zero.data(), d_out * 4, cudaMemcpyHostToDevice);
  *out = mlp;
  return DLMPC_OK;
}

extern "C" int64_t dlmpc_mlp_num_params(dlmpc_mlp *mlp) { return mlp ? mlp->n_params : -1; }

extern "C" int dlmpc_mlp_set_params(dlmpc_mlp *mlp, const float *params, int64_t n, const float *out_scale,
                                    const float *out_shift) {
  if (!mlp || !params || n != mlp->n_params) return mlp ? mlp->fail(DLMPC_ERR_ARG, "parameter count") : DLMPC_ERR_ARG;
  MK(cudaMemcpyAsync(mlp->w, params, n * 4, cudaMemcpyHostToDevice, mlp->stream), "H2D params");
  to_bf16_kernel<<<blocks_for(n), 256, 0, mlp->stream>>>(mlp->w, mlp->w_bf, n);
  if (out_scale) MK(cudaMemcpyAsync(mlp->scale, out_scale, mlp->d_out * 4, cudaMemcpyHostToDevice, mlp->stream), "H2D");
  if (out_shift) MK(cudaMemcpyAsync(mlp->shift, out_shift, mlp->d_out * 4, cudaMemcpyHostToDevice, mlp->stream), "H2D");
  MK(cudaMemsetAsync(mlp->m, 0, n * 4, mlp->stream), "memset");
  MK(cudaMemsetAsync(mlp->v, 0, n * 4, mlp->stream), "memset");
  mlp->step = 0;
  MK(cudaStreamSynchronize(mlp->stream), "set_params");
  return DLMPC_OK;
}

extern "C" int dlmpc_mlp_get_params(dlmpc_mlp *mlp, float *params, int64_t n) {
  if (!mlp || !params || n != mlp->n_params) return DLMPC_ERR_ARG;
  MK(cudaMemcpyAsync(params, mlp->w, n * 4, cudaMemcpyDeviceToHost, mlp->stream), "D2H params");
  MK(cudaStreamSynchronize(mlp->stream), "get_params");
  return DLMPC_OK;
}

namespace dlmpc {
// The stream the network's kernels run on (for callers that order it against
// their own stream).
cudaStream_t mlp_stream(const dlmpc_mlp *mlp) { return mlp->stream; }
}  // namespace dlmpc

extern "C" int dlmpc_mlp_forward(dlmpc_mlp *mlp, const float *x_dev, int32_t n, float *y_dev) {
  if (!mlp || !x_dev || !y_dev || n < 1) return DLMPC_ERR_ARG;
  return forward(mlp, x_dev, n, y_dev, true);
}

extern "C" int dlmpc_mlp_gradients(dlmpc_mlp *mlp, const float *x_dev, const float *t_dev, int32_t n, float *grad_host,
                                   double *loss_host) {
  if (!mlp || !x_dev || !t_dev || n < 1) return DLMPC_ERR_ARG;
  int rc = backward(mlp, x_dev, t_dev, n);
  if (rc) return rc;
  if (grad_host)
    MK(cudaMemcpyAsync(grad_host, mlp->grad, mlp->n_params * 4, cudaMemcpyDeviceToHost, mlp->stream), "D2H grad");
  if (loss_host) MK(cudaMemcpyAsync(loss_host, mlp->loss, 8, cudaMemcpyDeviceToHost, mlp->stream), "D2H loss");
  MK(cudaStreamSynchronize(mlp->stream), "gradients");
  if (loss_host) *loss_host /= (double)n * mlp->d_out;
  return DLMPC_OK;
}

extern "C" int dlmpc_mlp_train_step(dlmpc_mlp *mlp, const float *x_dev, const float *t_dev, int32_t n, float lr,
                                    float weight_decay, double *loss_host) {
  if (!mlp || !x_dev || !t_dev || n < 1) return DLMPC_ERR_ARG;
  int rc = backward(mlp, x_dev, t_dev, n);
  if (rc) return rc;
  const float b1 = 0.9f, b2 = 0.999f;
  mlp->step += 1;
  const float c1 = 1.f - powf(b1, (float)mlp->step), c2 = 1.f - powf(b2, (float)mlp->step);
  adamw_kernel<<<blocks_for(mlp->n_params), 256, 0, mlp->stream>>>(mlp->w, mlp->grad, mlp->m, mlp->v, mlp->w_bf,
                                                                   mlp->n_params, lr, b1, b2, 1e-8f, weight_decay, c1, c2);
  MK(cudaGetLastError(), "adamw_kernel");
  if (loss_host) {
    MK(cudaMemcpyAsync(loss_host, mlp->loss, 8, cudaMemcpyDeviceToHost, mlp->stream), "D2H loss");
    MK(cudaStreamSynchronize(mlp->stream), "train_step");
    *loss_host /= (double)n * mlp->d_out;
  }
  return DLMPC_OK;
}

extern "C" const char *dlmpc_mlp_last_error(dlmpc_mlp *mlp) { return mlp ? mlp->err.c_str() : ""; }

extern "C" void dlmpc_mlp_destroy(dlmpc_mlp *mlp) { delete mlp; }
