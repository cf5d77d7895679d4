// Line-solve kernels for float fields with the periodic correction evaluated
// to FP64 accuracy (LineCoef::wrap_ext: the psi operator's solves, whose wrap
// weight lam^n is far above FP32 resolution).
#include "ib_linesolve.cuh"

namespace ibg {
cudaError_t launch_sweep_f32_ext(int axis, int pro, int epi, int nfields, const SweepArgs<float> &a, cudaStream_t s,
                                 int cfg) {
  return launch_sweep_impl<float, true>(axis, pro, epi, nfields, a, s, cfg);
}
}  // namespace ibg
