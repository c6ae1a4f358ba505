// Host-side launch plans for the fused X-pass and the p-phase.
#pragma once
#include <cuda_runtime.h>

#include "pphase.cuh"
#include "xpass.cuh"

namespace relax {

// storage kinds of X (mirrors relax_dtype)
enum XKind : int { XK_F64 = 0, XK_F32 = 1, XK_BF16 = 2, XK_FP8 = 3 };

inline int xkind_esize(int xk) { return xk == XK_F64 ? 8 : xk == XK_F32 ? 4 : xk == XK_BF16 ? 2 : 1; }
inline int xkind_vec(int xk) { return 16 / xkind_esize(xk); }

struct XPlan {
  int xk = 0;           // storage of X
  bool vec_double = false;  // beta / y / partial storage is double (X in F64)
  bool cert = false;    // FP64 accumulation, 2 forward vectors
  int NF = 1, NB = 1;
  int NV = 2, R = 2, S = 2, C = 1;
  int64_t slice = 0;
  uint32_t slot_bytes = 0;
  size_t smem = 0;
  int ncl = 1;          // clusters launched
  const void* kernel = nullptr;
};

constexpr int XBLOCK = 224;  // consumer threads (7 warps) + 1 producer warp = 256

// Builds a plan (chooses NV, C, R, S; queries cluster occupancy).  Returns
// cudaErrorNotSupported when p is too large for one cluster of <= 16 CTAs.
cudaError_t xpass_plan(XPlan& pl, int xk, bool vec_double, bool cert, int NF, int NB, int64_t n,
                       int64_t p);
cudaError_t xpass_launch(const XPlan& pl, const XPassArgs& a, cudaStream_t st);

struct PPlan {
  const void* kernel = nullptr;
  int grid = 1;
  bool vdouble = false, gdouble = false;
};
cudaError_t pphase_plan(PPlan& pl, bool vdouble, bool gdouble, int64_t p);
cudaError_t pphase_launch(const PPlan& pl, const PArgs& a, cudaStream_t st);

}  // namespace relax
