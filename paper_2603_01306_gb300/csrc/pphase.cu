// Instantiations and cooperative launch of the p-phase kernel.
#include <algorithm>
#include <cstdlib>

#include "launch.cuh"

namespace relax {

cudaError_t pphase_plan(PPlan& pl, bool vdouble, int64_t p, bool backtrack, bool fast) {
  pl = PPlan{};
  pl.vdouble = vdouble;
  if (backtrack && !vdouble) return cudaErrorNotSupported;   // the loop's vectors are FP64
  if (fast && (backtrack || !vdouble)) return cudaErrorNotSupported;
  pl.kernel = backtrack ? reinterpret_cast<const void*>(&pphase_kernel<double, PEPT, true>)
              : fast    ? reinterpret_cast<const void*>(&pphase_kernel<double, PEPT, false, false, true>)
              : vdouble ? reinterpret_cast<const void*>(&pphase_kernel<double, PEPT>)
                        : reinterpret_cast<const void*>(&pphase_kernel<float, PEPT>);
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pl.kernel, PBLOCK, 0);
  if (e != cudaSuccess) return e;
  const int64_t maxgrid = (int64_t)nsm * std::max(per, 1);
  pl.maxgrid = (int)maxgrid;
  // one element per thread where the co-resident grid allows (measured at
  // p = 50000: 1 -> 0.080 ms per iteration, 2 -> 0.084, 4 -> 0.099: the
  // grid barriers cost less than the longer per-thread chains), at most
  // PEPT (RELAX_PP=e sets e elements per thread for tuning runs)
  int ept = 1;
  if (const char* ov = std::getenv("RELAX_PP")) ept = std::max(1, std::min(PEPT, std::atoi(ov)));
  const int64_t want = (p + (int64_t)ept * PBLOCK - 1) / ((int64_t)ept * PBLOCK);
  int64_t g = std::max<int64_t>(1, std::min<int64_t>(want, maxgrid));
  if (g * PBLOCK * PEPT < p) g = (p + (int64_t)PBLOCK * PEPT - 1) / ((int64_t)PBLOCK * PEPT);
  if (g > maxgrid) return cudaErrorNotSupported;
  pl.grid = (int)g;
  return cudaSuccess;
}

cudaError_t pphase_launch(const PPlan& pl, const PArgs& a, cudaStream_t st) {
  return pphase_launch_grid(pl, a, pl.grid, st);
}

cudaError_t pphase_launch_grid(const PPlan& pl, const PArgs& a, int grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(PBLOCK, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[1] = {(void*)&a};
  return cudaLaunchKernelExC(&cfg, pl.kernel, args);
}

// one cluster per problem: PEPT coordinates per thread (two CTAs fit an SM)
// on up to 16 CTAs (a non-portable cluster size), else PEPT_CLUSTER per
// thread on up to 8
static cudaError_t cluster_try(PPlan& pl, int64_t p, const void* kernel, int ept, int max_seg) {
  pl = PPlan{};
  pl.vdouble = true;
  pl.kernel = kernel;
  const int64_t seg = (p + (int64_t)PBLOCK * ept - 1) / ((int64_t)PBLOCK * ept);
  if (seg < 1 || seg > max_seg) return cudaErrorNotSupported;
  if (seg > 8) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cudaErrorNotSupported;
    }
  }
  pl.seg = (int)seg;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)seg;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)seg, 1, 1);
  cfg.blockDim = dim3(PBLOCK, 1, 1);
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, pl.kernel, &cfg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cudaErrorNotSupported;
  }
  if (nclusters < 1) return cudaErrorNotSupported;
  pl.maxgrid = nclusters * (int)seg;
  pl.grid = (int)seg;
  return cudaSuccess;
}

cudaError_t pphase_cluster_plan(PPlan& pl, int64_t p, bool backtrack, bool fast) {
  if (fast && backtrack) return cudaErrorNotSupported;
  const void* k4 = pphase_cluster_kernel(PEPT, backtrack, fast);
  const void* k8 = pphase_cluster_kernel(PEPT_CLUSTER, backtrack, fast);
  if (cluster_try(pl, p, k4, PEPT, 16) == cudaSuccess) return cudaSuccess;
  return cluster_try(pl, p, k8, PEPT_CLUSTER, 8);
}

cudaError_t pphase_launch_clusters(const PPlan& pl, const PArgs& a, int nseg, cudaStream_t st) {
  if (pl.seg < 1 || a.seg_blocks != pl.seg || !a.cluster || nseg < 1) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)pl.seg;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(nseg * pl.seg), 1, 1);
  cfg.blockDim = dim3(PBLOCK, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[1] = {(void*)&a};
  return cudaLaunchKernelExC(&cfg, pl.kernel, args);
}

}  // namespace relax
