// Launch planning for the fused X-pass and the p-phase.
#include <algorithm>

#include "launch.cuh"

namespace relax {

const void* xpass_ptr_f64(bool cert, int NF, int NB, int NV, int R);
const void* xpass_ptr_f32(bool cert, int NF, int NB, int NV, int R);
const void* xpass_ptr_bf16(bool cert, int NF, int NB, int NV, int R);
const void* xpass_ptr_fp8(bool cert, int NF, int NB, int NV, int R);

static const void* xpass_ptr(int xk, bool cert, int NF, int NB, int NV, int R) {
  switch (xk) {
    case XK_F64: return xpass_ptr_f64(cert, NF, NB, NV, R);
    case XK_F32: return xpass_ptr_f32(cert, NF, NB, NV, R);
    case XK_BF16: return xpass_ptr_bf16(cert, NF, NB, NV, R);
    case XK_FP8: return xpass_ptr_fp8(cert, NF, NB, NV, R);
    default: return nullptr;
  }
}

static int device_smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

cudaError_t xpass_plan(XPlan& pl, int xk, bool vec_double, bool cert, int NF, int NB, int64_t n,
                       int64_t p) {
  pl = XPlan{};
  pl.xk = xk;
  pl.vec_double = vec_double;
  pl.cert = cert;
  pl.NF = NF;
  pl.NB = NB;
  const int vec = xkind_vec(xk);
  const int es = xkind_esize(xk);
  int choices_f[3] = {2, 4, 8};
  int choices_bf[3] = {1, 2, 4};
  int choices_f8[2] = {1, 2};
  const int* ch = (xk == XK_BF16) ? choices_bf : (xk == XK_FP8) ? choices_f8 : choices_f;
  const int nch = (xk == XK_FP8) ? 2 : 3;
  int NV = -1, C = 0;
  for (int pass = 0; pass < 2 && NV < 0; ++pass) {
    const int cmax = pass == 0 ? 8 : 16;
    for (int i = 0; i < nch; ++i) {
      const int64_t per = (int64_t)XBLOCK * ch[i] * vec;
      const int64_t c = (p + per - 1) / per;
      if (c <= cmax) { NV = ch[i]; C = (int)c; break; }
    }
  }
  if (NV < 0) return cudaErrorNotSupported;
  if (cert && xk != XK_F64 && xk != XK_F32) return cudaErrorNotSupported;
  // slice: columns per rank, a multiple of the vector width, ranks cover [0, p)
  int64_t slice = (p + C - 1) / C;
  slice = (slice + vec - 1) / vec * vec;
  while (C > 1 && (int64_t)(C - 1) * slice >= p) --C;
  pl.NV = NV;
  pl.C = C;
  pl.slice = slice;
  pl.slot_bytes = (uint32_t)(((slice * es) + 15) / 16 * 16);
  pl.R = pl.slot_bytes >= 8192 ? 2 : 8;
  const int smax = device_smem_optin();
  const int ta = cert ? 8 : (vec_double ? 8 : 4);
  const size_t misc = 1024 + (size_t)4 * C * pl.R * NF * ta + (size_t)2 * (XBLOCK / 32) * pl.R * NF * ta;
  int S = (int)((smax - (int)misc - 256) / ((size_t)pl.R * pl.slot_bytes));
  S = std::min(S, 8);
  if (S < 2) return cudaErrorNotSupported;
  pl.S = S;
  pl.smem = (size_t)S * pl.R * pl.slot_bytes + (size_t)(2 * S + 4) * 8 + (size_t)4 * C * pl.R * NF * ta +
            (size_t)2 * (XBLOCK / 32) * pl.R * NF * ta;
  pl.kernel = xpass_ptr(xk, cert, NF, NB, NV, pl.R);
  if (!pl.kernel) return cudaErrorNotSupported;
  cudaError_t e = cudaFuncSetAttribute(pl.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(pl.kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(XBLOCK + 32, 1, 1);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int maxcl = 0;
  e = cudaOccupancyMaxActiveClusters(&maxcl, pl.kernel, &cfg);
  if (e != cudaSuccess) return e;
  if (maxcl < 1) return cudaErrorNotSupported;
  const int64_t ntiles = (n + pl.R - 1) / pl.R;
  pl.ncl = (int)std::min<int64_t>(maxcl, std::max<int64_t>(ntiles, 1));
  return cudaSuccess;
}

cudaError_t xpass_launch(const XPlan& pl, const XPassArgs& a, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = pl.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(pl.C * pl.ncl, 1, 1);
  cfg.blockDim = dim3(XBLOCK + 32, 1, 1);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[1] = {(void*)&a};
  return cudaLaunchKernelExC(&cfg, pl.kernel, args);
}

}  // namespace relax
