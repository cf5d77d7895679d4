// Line-solve kernels instantiated for double fields.
#include "ib_linesolve.cuh"

namespace ibg {
template <>
cudaError_t launch_sweep<double>(int axis, int pro, int epi, int nfields, const SweepArgs<double> &a, cudaStream_t s,
                               int cfg) {
  return launch_sweep_impl<double, false>(axis, pro, epi, nfields, a, s, cfg);
}
}  // namespace ibg
