// Line-solve kernels instantiated for float fields.
#include "ib_linesolve.cuh"

namespace ibg {
template <>
cudaError_t launch_sweep<float>(int axis, int pro, int epi, int nfields, const SweepArgs<float> &a, cudaStream_t s) {
  return launch_sweep_impl<float>(axis, pro, epi, nfields, a, s);
}
}  // namespace ibg
