// Instantiations, plan and launch of the strip-stationary fused pass.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstdlib>

#include "launch.cuh"

namespace relax {

template <typename TX, typename TA, int NF, int NB, bool FF = false>
static const void* kptr() {
  return reinterpret_cast<const void*>(&xstrip_kernel<TX, TA, NF, NB, FF>);
}

static const void* xstrip_ptr(int xk, bool f64acc, int NF, int NB) {
  if (NF == 1 && NB == 1) {
    if (xk == XK_F64) return kptr<double, double, 1, 1>();
    // FP32 X: the certificate / power-iteration pass in float-float arithmetic
    if (xk == XK_F32) return f64acc ? kptr<float, float, 1, 1, true>() : kptr<float, float, 1, 1>();
    if (xk == XK_BF16 && !f64acc) return kptr<__nv_bfloat16, float, 1, 1>();
    if (xk == XK_FP8 && !f64acc) return kptr<__nv_fp8_e4m3, float, 1, 1>();
  } else if (NF == 1 && NB == 2 && f64acc) {
    // the logistic loop's float-float pass; the two-dual-point certificate
    if (xk == XK_F32) return kptr<float, float, 1, 2, true>();
    if (xk == XK_F64) return kptr<double, double, 1, 2>();
  } else if (NF == 1 && NB == 2 && !f64acc) {
    if (xk == XK_F64) return kptr<double, double, 1, 2>();
    if (xk == XK_F32) return kptr<float, float, 1, 2>();
    if (xk == XK_BF16) return kptr<__nv_bfloat16, float, 1, 2>();
    if (xk == XK_FP8) return kptr<__nv_fp8_e4m3, float, 1, 2>();
  } else if (NF == 2 && NB == 1) {
    if (xk == XK_F64) return kptr<double, double, 2, 1>();
    if (xk == XK_F32 && f64acc) return kptr<float, float, 2, 1, true>();
  }
  return nullptr;
}

static int xs_tv(int vec) { return vec == 2 ? 6 : vec == 4 ? 6 : vec == 8 ? 3 : 2; }   // XSShape<VEC>::TV

// Shape of the pass for an n x p design.
//  * strips of a row of at most 32*TV vectors (the registers of one lane
//    row), chosen to keep the most SMs busy (Gc strips x Gr row groups), at
//    least 2 KB wide where possible;
//  * a strip is nbox tensor boxes of `inner` <= 256 columns;
//  * blocks of B <= 16 rows so that a stage is about 40 KB; 3 + 3 warps and
//    as many stages per warp as shared memory holds (ring A first);
//  * phase A may lead phase B by `lag` blocks: about 64 MB of X in L2 (at
//    least 20 blocks with four or more row groups).
// RELAX_XS="B,SA,SB,lag,vps,mA,mB" overrides for tuning runs (0 keeps a default).
cudaError_t xstrip_plan(XSPlan& pl, int xk, bool f64acc, int NF, int NB, int64_t n, int64_t p) {
  pl = XSPlan{};
  pl.xk = xk;
  pl.cert = f64acc;
  pl.NF = NF;
  pl.NB = NB;
  pl.kernel = xstrip_ptr(xk, f64acc, NF, NB);
  if (!pl.kernel || n < 1 || p < 1 || n > INT32_MAX || p > INT32_MAX) return cudaErrorNotSupported;
  int dev = 0, nsm = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int es = xkind_esize(xk);
  const int vec = xkind_vec(xk);
  int B_f = 0, SA_f = 0, SB_f = 0, lag_f = 0, vps_f = 0, mA_f = 0, mB_f = 0;
  if (const char* ov = std::getenv("RELAX_XS"))
    std::sscanf(ov, "%d,%d,%d,%d,%d,%d,%d", &B_f, &SA_f, &SB_f, &lag_f, &vps_f, &mA_f, &mB_f);
  // strips: over the number of row groups Gr, the strip width (at most `cap`
  // vectors) that keeps the most SMs busy, strips under 2 KB counted as
  // streaming less efficiently
  const int64_t nvec = (p + vec - 1) / vec;
  const int64_t cap = (int64_t)32 * xs_tv(vec);
  int64_t vps = 0;
  double best = -1.0;
  for (int64_t gr = 1; gr <= nsm; ++gr) {
    int64_t gc = std::min<int64_t>(nsm / gr, nvec);
    if (gc < 1) break;
    const int64_t v = (nvec + gc - 1) / gc;
    if (v > cap) continue;
    gc = (nvec + v - 1) / v;
    if (gr > 1 && n < gr * 16) break;   // too few rows to keep the groups busy
    const double score = (double)(gc * gr) * std::sqrt(std::min(1.0, (double)(v * 16) / 2048.0));
    if (score > best * 1.0001) { best = score; vps = v; }
  }
  if (vps_f > 0) vps = vps_f;
  if (vps <= 0 || vps > cap) return cudaErrorNotSupported;   // p wider than nsm strips of one lane row
  const int64_t cols = vps * vec;
  const int64_t nbox = (cols + 255) / 256;
  const int64_t inner = ((cols + nbox - 1) / nbox + vec - 1) / vec * vec;
  pl.inner = (int)inner;
  pl.nbox = (int)nbox;
  pl.sw = nbox * inner;
  if (pl.sw / vec > cap) return cudaErrorNotSupported;
  const int64_t Gc = (p + pl.sw - 1) / pl.sw;
  pl.Gc = (int)Gc;
  // blocks
  int64_t B = std::max<int64_t>(1, std::min<int64_t>(XS_MAXB, 40960 / (pl.sw * es)));
  if (B_f > 0) B = std::min<int64_t>(B_f, XS_MAXB);
  B = std::min<int64_t>(B, n);
  auto boxb = [&](int64_t b) { return (b * inner * es + 127) / 128 * 128; };
  const size_t fixed = 2048 + 128;   // static shared memory, alignment slack
  auto fits = [&](int64_t b, int sa, int sb) {
    return (size_t)(sa + sb) * (size_t)(nbox * boxb(b)) + fixed <= (size_t)optin;
  };
  while (B > 1 && !fits(B, 3, 3)) --B;
  int SA = 3, SB = 3;   // 2 + SA + SB warps <= 8
  if (SA_f > 0) SA = std::min(SA_f, XS_MAXS);
  if (SB_f > 0) SB = std::min(SB_f, XS_MAXS);
  if (2 + SA + SB > XS_MAXT / 32 || !fits(B, SA, SB)) return cudaErrorNotSupported;
  // ring depths: stages per warp.  A stage is held from its TMA issue until
  // its warp has read the block, so small blocks (narrow element types) need
  // more of them to keep enough of X in flight; ring A (HBM) first, then
  // ring B (L2), while shared memory allows
  int mA = 1, mB = 1;
  if (mA_f > 0 || mB_f > 0) {
    mA = std::max(1, mA_f);
    mB = std::max(1, mB_f);
  } else {
    while ((mA + 1) * SA <= XS_MAXR && fits(B, (mA + 1) * SA, mB * SB)) ++mA;
    if (mA > 1 && (mB + 1) * SB <= XS_MAXR && fits(B, mA * SA, (mB + 1) * SB)) ++mB;
  }
  if (mA * SA > XS_MAXR || mB * SB > XS_MAXR || !fits(B, mA * SA, mB * SB)) return cudaErrorNotSupported;
  pl.RA = mA * SA;
  pl.RB = mB * SB;
  pl.B = (int)B;
  pl.boxb = (int)boxb(B);
  pl.nblk = (int)((n + B - 1) / B);
  pl.SA = SA;
  pl.SB = SB;
  pl.Gr = (int)std::max<int64_t>(1, std::min<int64_t>(nsm / Gc, pl.nblk));
  const double row_bytes = (double)p * es;
  pl.lag = lag_f > 0 ? lag_f : (int)std::max(4.0, std::min(64.0, 64.0e6 / (B * row_bytes * pl.Gr)));
  // tall designs (four or more row groups): a deeper lead measured faster
  // (100000 x 20000 logistic: lag 12 -> 20 took the pass from 0.28 to 0.43 of
  // the copy bandwidth) although it holds more of X than L2 does
  if (lag_f <= 0 && pl.Gr >= 4) pl.lag = std::max(pl.lag, 20);
  pl.grid = pl.Gc * pl.Gr;
  pl.threads = 32 * (2 + SA + SB);   // two producers, SA dot, SB axpy
  // the combine of the axpy warps' strip sums reuses the rings
  const size_t ring = (size_t)(pl.RA + pl.RB) * nbox * pl.boxb;
  const size_t comb = (size_t)SB * NB * pl.sw * sizeof(double);
  pl.smem = std::max(ring, comb) + 128;
  if (pl.smem + 2048 > (size_t)optin) return cudaErrorNotSupported;
  // the attribute belongs to the kernel, shared by every plan and handle: only raise it
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, pl.kernel);
  if (e != cudaSuccess) return e;
  if (fa.maxDynamicSharedSizeBytes < (int)pl.smem) {
    e = cudaFuncSetAttribute(pl.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    if (e != cudaSuccess) return e;
  }
  int per = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pl.kernel, pl.threads, pl.smem);
  if (e != cudaSuccess) return e;
  if (per < 1 || per * nsm < pl.grid) return cudaErrorNotSupported;
  return cudaSuccess;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  }
  return fn;
}

cudaError_t xstrip_bind(XSPlan& pl, const void* X, int64_t ldx, int64_t n, int64_t p) {
  const int es = xkind_esize(pl.xk);
  if ((reinterpret_cast<uintptr_t>(X) & 15u) != 0 || ((size_t)ldx * es) % 16 != 0 || ldx < p)
    return cudaErrorInvalidValue;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const CUtensorMapDataType dt = pl.xk == XK_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                 : pl.xk == XK_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : pl.xk == XK_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                    : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  const cuuint64_t dims[2] = {(cuuint64_t)p, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)ldx * es};
  const cuuint32_t box[2] = {(cuuint32_t)pl.inner, (cuuint32_t)pl.B};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(&pl.tm, dt, 2, const_cast<void*>(X), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// The per-pass area zeroed before every launch:
//   cnt[nblk] | zcnt | zmax[2] | zfix[NF][n]
static size_t zero_off_zcnt(const XSPlan& pl) { return ((size_t)pl.nblk * sizeof(unsigned) + 15) / 16 * 16; }
size_t xstrip_zero_bytes(const XSPlan& pl, int64_t n) {
  return zero_off_zcnt(pl) + 32 + (size_t)pl.NF * n * sizeof(unsigned long long);
}
void xstrip_zero_layout(const XSPlan& pl, void* base, XSArgs& a) {
  unsigned char* b = static_cast<unsigned char*>(base);
  const size_t oz = zero_off_zcnt(pl);
  a.cnt = reinterpret_cast<unsigned*>(b);
  a.zcnt = reinterpret_cast<unsigned*>(b + oz);
  a.zmax = reinterpret_cast<unsigned long long*>(b + oz + 16);
  a.zfix = reinterpret_cast<unsigned long long*>(b + oz + 32);
}

cudaError_t xstrip_launch(const XSPlan& pl, const XSArgs& a, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(a.cnt, 0, xstrip_zero_bytes(pl, a.n), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.gridDim = dim3(pl.grid, 1, 1);
  cfg.blockDim = dim3(pl.threads, 1, 1);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[1] = {(void*)&a};
  return cudaLaunchKernelExC(&cfg, pl.kernel, args);
}

}  // namespace relax
