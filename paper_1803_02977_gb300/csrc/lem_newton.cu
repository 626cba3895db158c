// lem_newton.cu -- Alg 6 (Step 7, Calculate Erosion) for a general slope
// exponent n-hat: Alg 5's uplift of the cells without receiver, then the
// Newton-Raphson solve of every cell's implicit update (erode_newton), level 1
// upward over the device-wide levels that the step kernel's stage phases
// computed.  One cooperative launch, one bounded grid barrier per wide level
// and runs of narrow levels in block 0 (phase_global_erode).  It is a kernel
// of its own, in its own translation unit, so that the n-hat = 1 step kernel
// is compiled exactly as without it.
#include <cuda_runtime.h>

#include "lem.h"
#include "lem_context.cuh"

namespace lem {

template <typename HT, typename CT>
__global__ void __launch_bounds__(kBD, 1)
    newton_erode_kernel(const __grid_constant__ StepArgs<HT, CT> a) {
  // L was stored by the levels phase (Alg 3) of an earlier launch
  const int L = ld_volatile(&a.st->nlevels);
  phase_global_erode<HT, CT, true>(a, L);
}

}  // namespace lem

// Launch the sweep for the step arguments of a context (lem_api.cu builds
// them); grid = the context's co-resident block count.
template <typename HT, typename CT>
int lem_newton_launch(const lem::StepArgs<HT, CT>& a, int grid, cudaStream_t stream) {
  void* args[] = {(void*)&a};
  const cudaError_t e = cudaLaunchCooperativeKernel(
      (const void*)&lem::newton_erode_kernel<HT, CT>, dim3(grid), dim3(lem::kBD), args, 0, stream);
  if (e == cudaSuccess) return LEM_OK;
  return e == cudaErrorMemoryAllocation ? LEM_ENOMEM : LEM_ECUDA;
}

template int lem_newton_launch<double, int>(const lem::StepArgs<double, int>&, int, cudaStream_t);
template int lem_newton_launch<double, long long>(const lem::StepArgs<double, long long>&, int,
                                                  cudaStream_t);
template int lem_newton_launch<float, int>(const lem::StepArgs<float, int>&, int, cudaStream_t);
template int lem_newton_launch<float, long long>(const lem::StepArgs<float, long long>&, int,
                                                 cudaStream_t);
