// Instantiations of the p-phase kernel for the cluster-per-problem launch of
// batched node solves (a translation unit of their own: compiled in parallel
// with the grid instantiations).
#include "launch.cuh"

namespace relax {

const void* pphase_cluster_kernel(int ept, bool backtrack, bool fast) {
  if (ept == PEPT)
    return backtrack ? reinterpret_cast<const void*>(&pphase_kernel<double, PEPT, true, true>)
           : fast    ? reinterpret_cast<const void*>(&pphase_kernel<double, PEPT, false, true, true>)
                     : reinterpret_cast<const void*>(&pphase_kernel<double, PEPT, false, true>);
  return backtrack ? reinterpret_cast<const void*>(&pphase_kernel<double, PEPT_CLUSTER, true, true>)
         : fast    ? reinterpret_cast<const void*>(&pphase_kernel<double, PEPT_CLUSTER, false, true, true>)
                   : reinterpret_cast<const void*>(&pphase_kernel<double, PEPT_CLUSTER, false, true>);
}

}  // namespace relax
