// Batched line-solve kernels (one launch over the grids of an ensemble size
// class) for float fields with the FP64-accurate periodic correction.
#include "ib_linesolve.cuh"

namespace ibg {
cudaError_t launch_sweep_batch_f32_ext(int axis, int pro, int epi, int nfields, const SweepArgs<float> *a, int n,
                                       cudaStream_t s, int cfg) {
  return launch_sweep_batch_impl<float, true>(axis, pro, epi, nfields, a, n, s, cfg);
}
}  // namespace ibg
