// Batched line-solve kernels (one launch over the grids of an ensemble size
// class) instantiated for double fields.
#include "ib_linesolve.cuh"

namespace ibg {
template <>
cudaError_t launch_sweep_batch<double>(int axis, int pro, int epi, int nfields, const SweepArgs<double> *a, int n,
                                       cudaStream_t s, int cfg) {
  return launch_sweep_batch_impl<double, false>(axis, pro, epi, nfields, a, n, s, cfg);
}
}  // namespace ibg
