// Instantiations of the fused X-pass for X stored as float (generated list).
#include "xpass.cuh"

namespace relax {

template <int NF, int NB, int NV, int R, typename TA>
static const void* pick() {
  return reinterpret_cast<const void*>(&xpass_kernel<float, float, TA, NF, NB, 224, NV, R>);
}

const void* xpass_ptr_f32(bool cert, int NF, int NB, int NV, int R) {
  if (!cert && NF == 1 && NB == 1 && NV == 2 && R == 2) return pick<1, 1, 2, 2, float>();
  if (!cert && NF == 1 && NB == 2 && NV == 2 && R == 2) return pick<1, 2, 2, 2, float>();
  if (!cert && NF == 1 && NB == 1 && NV == 2 && R == 8) return pick<1, 1, 2, 8, float>();
  if (!cert && NF == 1 && NB == 2 && NV == 2 && R == 8) return pick<1, 2, 2, 8, float>();
  if (cert && NF == 2 && NB == 1 && NV == 2 && R == 2) return pick<2, 1, 2, 2, double>();
  if (!cert && NF == 1 && NB == 1 && NV == 4 && R == 2) return pick<1, 1, 4, 2, float>();
  if (!cert && NF == 1 && NB == 2 && NV == 4 && R == 2) return pick<1, 2, 4, 2, float>();
  if (!cert && NF == 1 && NB == 1 && NV == 4 && R == 8) return pick<1, 1, 4, 8, float>();
  if (!cert && NF == 1 && NB == 2 && NV == 4 && R == 8) return pick<1, 2, 4, 8, float>();
  if (cert && NF == 2 && NB == 1 && NV == 4 && R == 2) return pick<2, 1, 4, 2, double>();
  if (!cert && NF == 1 && NB == 1 && NV == 8 && R == 2) return pick<1, 1, 8, 2, float>();
  if (!cert && NF == 1 && NB == 2 && NV == 8 && R == 2) return pick<1, 2, 8, 2, float>();
  if (!cert && NF == 1 && NB == 1 && NV == 8 && R == 8) return pick<1, 1, 8, 8, float>();
  if (!cert && NF == 1 && NB == 2 && NV == 8 && R == 8) return pick<1, 2, 8, 8, float>();
  if (cert && NF == 2 && NB == 1 && NV == 8 && R == 2) return pick<2, 1, 8, 2, double>();
  return nullptr;
}

}  // namespace relax
