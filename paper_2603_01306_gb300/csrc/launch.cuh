// Host-side launch plans for the fused pass over X and the p-phase.
#pragma once
#include <cuda_runtime.h>

#include "pphase.cuh"
#include "xstrip.cuh"
#include "xpass.cuh"

namespace relax {

// storage kinds of X (mirrors relax_dtype)
enum XKind : int { XK_F64 = 0, XK_F32 = 1, XK_BF16 = 2, XK_FP8 = 3 };

inline int xkind_esize(int xk) { return xk == XK_F64 ? 8 : xk == XK_F32 ? 4 : xk == XK_BF16 ? 2 : 1; }
inline int xkind_vec(int xk) { return 16 / xkind_esize(xk); }

// Strip-stationary fused pass (xstrip.cuh)
struct XSPlan {
  CUtensorMap tm{};        // the plan's X as a tensor (set by xstrip_bind)
  int xk = 0;
  bool cert = false;       // FP64 accumulation (certification / power iteration of FP32 data)
  int NF = 1, NB = 1;
  int Gc = 1, Gr = 1;      // column strips x row groups
  int64_t sw = 0;          // strip columns = nbox * inner
  int inner = 1, nbox = 1, boxb = 128;
  int B = 1, nblk = 1;     // rows per block, blocks
  int SA = 3, SB = 3, lag = 4;
  int RA = 3, RB = 3;       // ring stages, multiples of SA / SB
  int grid = 1, threads = 32;
  size_t smem = 0;
  const void* kernel = nullptr;
};
cudaError_t xstrip_plan(XSPlan& pl, int xk, bool f64acc, int NF, int NB, int64_t n, int64_t p);
// encode the plan's tensor map of X (16-byte aligned, ldx * size a multiple of 16)
cudaError_t xstrip_bind(XSPlan& pl, const void* X, int64_t ldx, int64_t n, int64_t p);
// The per-pass area (block counters, the grid's max |beta|, z in fixed point)
// starts at a.cnt; xstrip_launch zeroes it on the stream before the launch.
size_t xstrip_zero_bytes(const XSPlan& pl, int64_t n);
void xstrip_zero_layout(const XSPlan& pl, void* base, XSArgs& a);   // sets a.cnt, a.zcnt, a.zmax, a.zfix
cudaError_t xstrip_launch(const XSPlan& pl, const XSArgs& a, cudaStream_t st);

struct PPlan {
  const void* kernel = nullptr;
  int grid = 1;
  int maxgrid = 1;         // CTAs that can be co-resident (cooperative launches)
  bool vdouble = false;
  int seg = 0;             // cluster plans: CTAs per problem (the cluster size)
};
// backtrack: the instantiation with the backtracking step rule (FP64 vectors);
// fast: the loop's FP32 per-coordinate instantiation (FP32 data, fixed step)
cudaError_t pphase_plan(PPlan& pl, bool vdouble, int64_t p, bool backtrack = false, bool fast = false);
cudaError_t pphase_launch(const PPlan& pl, const PArgs& a, cudaStream_t st);
// the same kernel on `grid` CTAs (a segmented launch: grid = segments x a.seg_blocks <= maxgrid)
cudaError_t pphase_launch_grid(const PPlan& pl, const PArgs& a, int grid, cudaStream_t st);
// Batched p-phase of many problems of length p, each on one thread-block
// cluster of pl.seg CTAs: PEPT coordinates per thread on up to 16 CTAs where
// the device allows that non-portable cluster size, else PEPT_CLUSTER on up to
// 8; cudaErrorNotSupported when p needs more.
cudaError_t pphase_cluster_plan(PPlan& pl, int64_t p, bool backtrack = false, bool fast = false);
// the cluster instantiation with `ept` coordinates per thread (PEPT or PEPT_CLUSTER)
const void* pphase_cluster_kernel(int ept, bool backtrack, bool fast);
// nseg clusters (a.seg_blocks = pl.seg, a.cluster = 1); no co-residency needed
cudaError_t pphase_launch_clusters(const PPlan& pl, const PArgs& a, int nseg, cudaStream_t st);

}  // namespace relax
