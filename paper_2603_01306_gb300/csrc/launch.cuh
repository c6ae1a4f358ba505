// Host-side launch plans for the fused pass over X and the p-phase.
#pragma once
#include <cuda_runtime.h>

#include "pphase.cuh"
#include "xblock.cuh"
#include "xpass.cuh"

namespace relax {

// storage kinds of X (mirrors relax_dtype)
enum XKind : int { XK_F64 = 0, XK_F32 = 1, XK_BF16 = 2, XK_FP8 = 3 };

inline int xkind_esize(int xk) { return xk == XK_F64 ? 8 : xk == XK_F32 ? 4 : xk == XK_BF16 ? 2 : 1; }
inline int xkind_vec(int xk) { return 16 / xkind_esize(xk); }

// Fused pass by L2 row blocking (xblock.cuh)
struct XBPlan {
  int xk = 0;
  bool cert = false;       // FP64 accumulation (certification / power iteration of FP64 data)
  int NF = 1, NB = 1;
  int64_t cw = 0;          // chunk columns
  int nchunk = 1;
  int B = 1, nblk = 1, lag = 2;
  int64_t sw = 0;          // strip columns per CTA
  int beta_smem = 0;
  int grid = 1;
  size_t smem = 0;
  const void* kernel = nullptr;
};
cudaError_t xblock_plan(XBPlan& pl, int xk, bool f64acc, int NF, int NB, int64_t n, int64_t p);
// counters (2 * nblk unsigned) are zeroed on the stream before the launch
cudaError_t xblock_launch(const XBPlan& pl, const XBArgs& a, cudaStream_t st);

struct PPlan {
  const void* kernel = nullptr;
  int grid = 1;
  bool vdouble = false;
};
cudaError_t pphase_plan(PPlan& pl, bool vdouble, int64_t p);
cudaError_t pphase_launch(const PPlan& pl, const PArgs& a, cudaStream_t st);

}  // namespace relax
