// Persistent ADMM sweep (the kernel itself is in dlmpc_sweep.cuh): the
// instantiations for CTAs of up to 1024 threads (64 registers per thread),
// the dispatch to them or to the 768- and 896-thread tiers
// (dlmpc_sweep_t768.cu, 80 registers per thread; dlmpc_sweep_t896.cu, 72),
// and the host-side launch helpers.
#include "dlmpc_sweep.cuh"

namespace dlmpc {

const void *sweep_kernel_ptr_t768(int nx, int gt, bool blk);
const void *sweep_kernel_ptr_t896(int nx, int gt, bool blk);

template <int NX, int GT, bool BLK>
static const void *sweep_fn() {
  return reinterpret_cast<const void *>(&sweep_kernel<NX, GT, BLK, 1024>);
}

// blk: the full-cost-block variant, built for 64 and 128 threads per group;
// `threads` (gt * groups per CTA) picks the register tier
const void *sweep_kernel_ptr(int nx, int gt, bool blk, int threads) {
  if (threads <= 768) return sweep_kernel_ptr_t768(nx, gt, blk);
  if (threads <= 896) return sweep_kernel_ptr_t896(nx, gt, blk);
#define DLMPC_SWEEP_CASE(NXV)                                 \
  case NXV:                                                   \
    if (blk) {                                                \
      if (gt == 64) return sweep_fn<NXV, 64, true>();         \
      if (gt == 128) return sweep_fn<NXV, 128, true>();       \
      return nullptr;                                         \
    }                                                         \
    if (gt == 64) return sweep_fn<NXV, 64, false>();          \
    if (gt == 96) return sweep_fn<NXV, 96, false>();          \
    if (gt == 128) return sweep_fn<NXV, 128, false>();        \
    if (gt == 256) return sweep_fn<NXV, 256, false>();        \
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

int sweep_group_floats(int nx, int nu, int gt, int wave, int max_dcol, int max_dred_pad, int max_kpad, int max_nmem,
                       bool rows_cached) {
  return group_layout(nx, nu, gt, wave, max_dcol, max_dred_pad, max_kpad, max_nmem, rows_cached).total;
}

cudaError_t launch_sweep(const Params &P, int gt, int grid, size_t smem, cudaStream_t s) {
  const void *fn = sweep_kernel_ptr(P.nx, gt, P.block_cost != 0, gt * P.ng);
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
