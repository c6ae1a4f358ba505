// Instantiations of the fused X-pass for X stored as __nv_fp8_e4m3 (generated list).
#include "xpass.cuh"

namespace relax {

template <int NF, int NB, int NV, int R, typename TA>
static const void* pick() {
  return reinterpret_cast<const void*>(&xpass_kernel<__nv_fp8_e4m3, float, TA, NF, NB, 224, NV, R>);
}

const void* xpass_ptr_fp8(bool cert, int NF, int NB, int NV, int R) {
  if (!cert && NF == 1 && NB == 1 && NV == 1 && R == 2) return pick<1, 1, 1, 2, float>();
  if (!cert && NF == 1 && NB == 2 && NV == 1 && R == 2) return pick<1, 2, 1, 2, float>();
  if (!cert && NF == 1 && NB == 1 && NV == 1 && R == 8) return pick<1, 1, 1, 8, float>();
  if (!cert && NF == 1 && NB == 2 && NV == 1 && R == 8) return pick<1, 2, 1, 8, float>();
  if (!cert && NF == 1 && NB == 1 && NV == 2 && R == 2) return pick<1, 1, 2, 2, float>();
  if (!cert && NF == 1 && NB == 2 && NV == 2 && R == 2) return pick<1, 2, 2, 2, float>();
  if (!cert && NF == 1 && NB == 1 && NV == 2 && R == 8) return pick<1, 1, 2, 8, float>();
  if (!cert && NF == 1 && NB == 2 && NV == 2 && R == 8) return pick<1, 2, 2, 8, float>();
  return nullptr;
}

}  // namespace relax
