// Line-solve kernels instantiated for float fields.
#include "ib_linesolve.cuh"

namespace ibg {
// Plain load/store solves of y and z lines take the TMA kernel when it
// applies and the configuration asks for it (kTmaCfg) or is left to the
// library (cfg < 0); every other sweep takes the register kernels, with the
// FP64-accurate periodic correction where the coefficients ask for it
// (ib_sweep_f32_ext.cu).
template <>
cudaError_t launch_sweep<float>(int axis, int pro, int epi, int nfields, const SweepArgs<float> &a, cudaStream_t s,
                               int cfg) {
  if (axis != 0 && pro == PRO_LOAD && epi == EPI_STORE && (cfg < 0 || cfg == kTmaCfg) && sweep_tma_ok(a, axis))
    return launch_sweep_tma(axis, nfields, a, s);
  if (a.co.wrap_ext) return launch_sweep_f32_ext(axis, pro, epi, nfields, a, s, cfg);
  return launch_sweep_impl<float, false>(axis, pro, epi, nfields, a, s, cfg);
}
}  // namespace ibg

namespace ibg {
// candidate sweep configurations for the autotuner (ids of strided_cfg and,
// for FP32 rows of a multiple of 4 floats, kTmaCfg for axes 1, 2; x grid caps
// for axis 0)
int sweep_candidates(int axis, int nl, int nx, bool dbl, int *out, int max) {
  int k = 0;
  if (axis == 0) {
    for (int i = 0; i < kXCaps && k < max; ++i) out[k++] = i;
  } else {
    for (int i = 0; i < kStridedCfgs && k < max; ++i)
      if (strided_cfg_ok(i, nl, nx, dbl)) out[k++] = i;
    if (!dbl && nx % 4 == 0 && (nl <= 256 || nl % 2 == 0) && k < max) out[k++] = kTmaCfg;
  }
  return k;
}
void sweep_config_shape(int axis, int cfg, int nl, int *a, int *b, int *c) {
  if (axis == 0) {
    *a = 1;
    *b = 8;
    *c = xcap(cfg < 0 ? 1 : cfg);
  } else if (cfg == kTmaCfg) {
    *a = 1;
    sweep_tma_shape(nl, b, c);
  } else {
    const StridedCfg t = strided_cfg(cfg < 0 ? 0 : cfg);
    *a = t.vw;
    *b = t.ch;
    *c = t.w;
  }
}
}  // namespace ibg
