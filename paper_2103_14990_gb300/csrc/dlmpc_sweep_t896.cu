// The sweep kernel's instantiations for CTAs of 769 to 896 threads: 72
// registers per thread, so the iteration loop keeps its state in registers
// (the 1024-thread tier spills a few words at 64).  Separate translation unit
// so that the tiers compile in parallel.
#include "dlmpc_sweep.cuh"

namespace dlmpc {

template <int NX, int GT, bool BLK>
static const void *sweep_fn_t896() {
  return reinterpret_cast<const void *>(&sweep_kernel<NX, GT, BLK, 896>);
}

const void *sweep_kernel_ptr_t896(int nx, int gt, bool blk) {
#define DLMPC_SWEEP_CASE(NXV)                                   \
  case NXV:                                                     \
    if (blk) {                                                  \
      if (gt == 64) return sweep_fn_t896<NXV, 64, true>();      \
      if (gt == 128) return sweep_fn_t896<NXV, 128, true>();    \
      return nullptr;                                           \
    }                                                           \
    if (gt == 64) return sweep_fn_t896<NXV, 64, false>();       \
    if (gt == 96) return sweep_fn_t896<NXV, 96, false>();       \
    if (gt == 128) return sweep_fn_t896<NXV, 128, false>();     \
    if (gt == 256) return sweep_fn_t896<NXV, 256, false>();     \
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

}  // namespace dlmpc
