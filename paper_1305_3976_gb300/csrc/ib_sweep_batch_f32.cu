// Batched line-solve kernels (one launch over the grids of an ensemble size
// class) instantiated for float fields.
#include "ib_linesolve.cuh"

namespace ibg {
template <>
cudaError_t launch_sweep_batch<float>(int axis, int pro, int epi, int nfields, const SweepArgs<float> *a, int n,
                                      cudaStream_t s, int cfg) {
  if (n > 0 && a[0].co.wrap_ext) return launch_sweep_batch_f32_ext(axis, pro, epi, nfields, a, n, s, cfg);
  return launch_sweep_batch_impl<float, false>(axis, pro, epi, nfields, a, n, s, cfg);
}
}  // namespace ibg
