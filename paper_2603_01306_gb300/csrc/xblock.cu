// Instantiations, plan and launch of the L2-blocked fused pass.
#include <algorithm>
#include <cstdio>
#include <cstdlib>

#include "launch.cuh"

namespace relax {

template <typename TX, typename TA, int NF, int NB>
static const void* kptr() {
  return reinterpret_cast<const void*>(&xblock_kernel<TX, TA, NF, NB>);
}

static const void* xblock_ptr(int xk, bool f64acc, int NF, int NB) {
  if (NF == 1 && NB == 1) {
    if (xk == XK_F64) return kptr<double, double, 1, 1>();
    if (xk == XK_F32) return f64acc ? kptr<float, double, 1, 1>() : kptr<float, float, 1, 1>();
    if (xk == XK_BF16 && !f64acc) return kptr<__nv_bfloat16, float, 1, 1>();
    if (xk == XK_FP8 && !f64acc) return kptr<__nv_fp8_e4m3, float, 1, 1>();
  } else if (NF == 1 && NB == 2 && !f64acc) {
    if (xk == XK_F64) return kptr<double, double, 1, 2>();
    if (xk == XK_F32) return kptr<float, float, 1, 2>();
    if (xk == XK_BF16) return kptr<__nv_bfloat16, float, 1, 2>();
    if (xk == XK_FP8) return kptr<__nv_fp8_e4m3, float, 1, 2>();
  } else if (NF == 2 && NB == 1) {
    if (xk == XK_F64) return kptr<double, double, 2, 1>();
    if (xk == XK_F32 && f64acc) return kptr<float, double, 2, 1>();
  }
  return nullptr;
}

// Shape of the pass for an n x p design (RELAX_XB="B,nchunk,lag" overrides
// for tuning runs; 0 keeps a default).
cudaError_t xblock_plan(XBPlan& pl, int xk, bool f64acc, int NF, int NB, int64_t n, int64_t p) {
  pl = XBPlan{};
  pl.xk = xk;
  pl.cert = f64acc;
  pl.NF = NF;
  pl.NB = NB;
  pl.kernel = xblock_ptr(xk, f64acc, NF, NB);
  if (!pl.kernel) return cudaErrorNotSupported;
  int dev = 0, nsm = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int es = xkind_esize(xk);
  const int vec = xkind_vec(xk);
  const int ta = (xk == XK_F64 || f64acc) ? 8 : 4;
  int B_force = 0, nc_force = 0, lag_force = 0;
  if (const char* ov = std::getenv("RELAX_XB")) std::sscanf(ov, "%d,%d,%d", &B_force, &nc_force, &lag_force);
  // row blocks of about 12 MB; phase A may lead by `lag` blocks (L2 holds lag + 2)
  const double row_bytes = (double)p * es;
  int64_t B = (int64_t)std::max(8.0, std::min(1024.0, 12.0e6 / row_bytes));
  B = std::min<int64_t>(B, n);
  if (B_force > 0) B = std::min<int64_t>(B_force, n);
  pl.B = (int)B;
  pl.nblk = (int)((n + B - 1) / B);
  pl.lag = lag_force > 0 ? lag_force : std::max(1, (int)(60.0e6 / std::max(1.0, B * row_bytes)) - 2);
  pl.lag = std::min(pl.lag, 8);
  // chunks: enough work items in the lag window for every phase-A warp
  const int64_t nwA = (int64_t)nsm * XB_WA;
  const int64_t window = (int64_t)std::min(pl.nblk, pl.lag) * B;
  int64_t nchunk = std::max<int64_t>(1, (3 * nwA / 2 + window - 1) / std::max<int64_t>(window, 1));
  const int64_t max_chunk = std::max<int64_t>(1, (p + 32 * vec - 1) / (32 * vec));   // >= one vector per lane
  nchunk = std::min(nchunk, max_chunk);
  if (nc_force > 0) nchunk = nc_force;
  int64_t cw = (p + nchunk - 1) / nchunk;
  cw = (cw + vec - 1) / vec * vec;
  nchunk = (p + cw - 1) / cw;
  pl.cw = cw;
  pl.nchunk = (int)nchunk;
  // column strips: one per CTA, at most 4 vectors per lane of the 4 phase-B warps' width
  int64_t sw = (p + nsm - 1) / nsm;
  sw = (sw + vec - 1) / vec * vec;
  const int tv = vec >= 16 ? 1 : (vec >= 8 ? 2 : 4);   // XBShape<VEC>::TV
  if (sw > (int64_t)32 * tv * vec) return cudaErrorNotSupported;   // strip wider than phase B covers
  pl.sw = sw;
  pl.grid = (int)std::min<int64_t>(nsm, (p + sw - 1) / sw);
  if (pl.grid < 1) pl.grid = 1;
  // shared memory
  const size_t rbytes = ((size_t)NB * B * ta + 15) / 16 * 16;
  const size_t cbytes = (size_t)XB_WB * NB * sw * 8;
  const size_t pst = (size_t)(p + 15) / 16 * 16;
  const size_t bbytes = (size_t)NF * pst * ta + 64;
  pl.beta_smem = (bbytes + rbytes + cbytes + 1024 <= (size_t)optin) ? 1 : 0;
  pl.smem = (pl.beta_smem ? bbytes : 0) + rbytes + std::max<size_t>(cbytes, 64);
  cudaError_t e = cudaFuncSetAttribute(pl.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return e;
  int per = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pl.kernel, XB_THREADS, pl.smem);
  if (e != cudaSuccess) return e;
  if (per < 1 || per * nsm < pl.grid) return cudaErrorNotSupported;
  return cudaSuccess;
}

cudaError_t xblock_launch(const XBPlan& pl, const XBArgs& a, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(a.done, 0, sizeof(unsigned) * 2 * (size_t)pl.nblk, st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.gridDim = dim3(pl.grid, 1, 1);
  cfg.blockDim = dim3(XB_THREADS, 1, 1);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[1] = {(void*)&a};
  return cudaLaunchKernelExC(&cfg, pl.kernel, args);
}

}  // namespace relax
