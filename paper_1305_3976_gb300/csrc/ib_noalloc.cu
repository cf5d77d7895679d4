// ib_split_solve_noalloc: the direction-split line solve of ib_split_solve
// for callers that cannot allocate device memory.
//
// Who needs it: a host process whose device memory is owned by someone else
// (a framework's caching allocator, a fixed memory budget handed out at
// start-up) or a latency-critical loop that must not call cudaMalloc because
// it synchronises the whole device.  ib_split_solve allocates a small table of
// powers lam^k per (n, r) the first time it sees them; this variant keeps that
// table in a fixed array inside the library instead and allocates nothing.
//
// The scratch: one file-scope __device__ array of 2 x 3 x (IB_NOALLOC_MAX_N + 8)
// doubles (about 25 KB).  Every GPU that loads the library holds it until the
// process exits.  Host code cannot use the array's name as a device address,
// so the first call on each device looks the address up with
// cudaGetSymbolAddress while that device is current and caches it (again
// whenever the device's context has changed since).  Devices 0 .. 63 are
// supported.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/ib_gb300.h"
#include "ib_internal.cuh"

using namespace ibg;

namespace {

constexpr int kMaxN = IB_NOALLOC_MAX_N;
constexpr int kRow = kMaxN + 8;  // one table of lam^0 .. lam^n per axis
constexpr int kMaxDevices = 64;

// [0][axis][k]: FP64 table; [1][axis][...]: FP32 table in the first half of
// the row's bytes and the FP32 remainders lam^k - (float)lam^k in the second
// half.  Rewritten completely by every call.
static __device__ __align__(256) double g_noalloc_pw[2][3][kRow];

// per device: the context the address was looked up in, and the address.  A
// device whose primary context was destroyed and created again (for example
// after cudaDeviceReset) reloads the library's module, and the array may then
// sit at another address, so the lookup is repeated when the context changes.
std::mutex g_mu;
void *g_ctx[kMaxDevices] = {};
double *g_addr[kMaxDevices] = {};

// the current driver context (cuCtxGetCurrent, reached through the runtime's
// entry-point query so that the library needs no link against libcuda)
typedef int (*CtxGetCurrentFn)(void **);
CtxGetCurrentFn ctx_get_current() {
  static std::once_flag once;
  static CtxGetCurrentFn fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (CtxGetCurrentFn)p;
  });
  return fn;
}

// lam^k for k = 0..n of every axis; blockIdx.x = axis.  lam^k by binary
// powering in FP64, the FP32 table is the FP64 value rounded.
__global__ void k_fill_powers(double *base, int n0, int n1, int n2, double l0, double l1, double l2) {
  const int a = blockIdx.x;
  const int n = a == 0 ? n0 : (a == 1 ? n1 : n2);
  const double lam = a == 0 ? l0 : (a == 1 ? l1 : l2);
  double *pd = base + (size_t)a * kRow;
  float *pf = reinterpret_cast<float *>(base + (size_t)(3 + a) * kRow);
  for (int k = threadIdx.x; k <= n; k += blockDim.x) {
    double p = 1.0, b = lam;
    for (int e = k; e > 0; e >>= 1) {
      if (e & 1) p *= b;
      b *= b;
    }
    pd[k] = p;
    pf[k] = (float)p;
    pf[kRow + k] = (float)(p - (double)(float)p);
  }
}

}  // namespace

// defined in ib_runtime.cu: records the message returned by ib_last_error()
int ib_internal_fail(int code, const char *msg);

extern "C" int ib_split_solve_noalloc(int precision, int dim, const int n[3], const double r[3], const void *f,
                                      void *psi, void *stream) {
  if (!n || !r || !f || !psi) return ib_internal_fail(IB_ERR_ARG, "ib_split_solve_noalloc: null argument");
  if (dim != 2 && dim != 3) return ib_internal_fail(IB_ERR_ARG, "ib_split_solve_noalloc: dim must be 2 or 3");
  if (precision != IB_FP32 && precision != IB_FP64)
    return ib_internal_fail(IB_ERR_ARG, "ib_split_solve_noalloc: precision");
  for (int a = 0; a < dim; ++a) {
    if (n[a] > kMaxN) {
      char buf[160];
      snprintf(buf, sizeof(buf), "ib_split_solve_noalloc: n[%d] = %d exceeds the fixed scratch limit of %d", a, n[a],
               kMaxN);
      return ib_internal_fail(IB_ERR_ARG, buf);
    }
    if (n[a] < 8) return ib_internal_fail(IB_ERR_ARG, "ib_split_solve_noalloc: n must be >= 8");
    if (!(r[a] >= 0)) return ib_internal_fail(IB_ERR_ARG, "ib_split_solve_noalloc: r must be >= 0");
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ib_internal_fail(IB_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return ib_internal_fail(IB_ERR_ARG, "ib_split_solve_noalloc: device index");
  CtxGetCurrentFn get_ctx = ctx_get_current();
  if (!get_ctx) return ib_internal_fail(IB_ERR_CUDA, "ib_split_solve_noalloc: cuCtxGetCurrent unavailable");
  double *base;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    void *ctx = nullptr;
    if (get_ctx(&ctx) != 0) return ib_internal_fail(IB_ERR_CUDA, "ib_split_solve_noalloc: cuCtxGetCurrent failed");
    if (!ctx || !g_addr[dev] || g_ctx[dev] != ctx) {
      // no context yet on this thread (the lookup below creates the device's
      // primary context), a first call, or a context created anew
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_pw);
      if (e != cudaSuccess) return ib_internal_fail(IB_ERR_CUDA, cudaGetErrorString(e));
      if (get_ctx(&ctx) != 0 || !ctx)
        return ib_internal_fail(IB_ERR_CUDA, "ib_split_solve_noalloc: no current CUDA context");
      g_addr[dev] = (double *)p;
      g_ctx[dev] = ctx;
    }
    base = g_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  double lam[3] = {0, 0, 0}, inv_c[3] = {1, 1, 1}, inv_1m[3] = {1, 1, 1};
  int nn[3] = {8, 8, 8};
  for (int a = 0; a < dim; ++a) {
    const double q = 1.0 + 2.0 * r[a] + sqrt(1.0 + 4.0 * r[a]);
    lam[a] = 2.0 * r[a] / q;
    inv_c[a] = 2.0 / q;
    double p = 1.0;
    for (int k = 0; k < n[a]; ++k) p *= lam[a];
    inv_1m[a] = 1.0 / (1.0 - p);
    nn[a] = n[a];
  }
  k_fill_powers<<<dim, 128, 0, s>>>(base, nn[0], nn[1], nn[2], lam[0], lam[1], lam[2]);
  e = cudaGetLastError();
  if (e != cudaSuccess) return ib_internal_fail(IB_ERR_CUDA, cudaGetErrorString(e));
  // the sweeps are linear: the last one applies the product of the 1/c
  double prod = 1.0;
  for (int a = 0; a < dim; ++a) prod *= inv_c[a];
  for (int a = 0; a < dim; ++a) {
    const double scale = a == dim - 1 ? prod : 1.0;
    if (precision == IB_FP32) {
      SweepArgs<float> sa;
      memset(&sa, 0, sizeof(sa));
      sa.f[0] = (float *)psi;
      sa.fin[0] = a == 0 ? (const float *)f : nullptr;
      for (int q = 0; q < 3; ++q) sa.n[q] = q < dim ? n[q] : 1;
      sa.dim = dim;
      const float *pf = reinterpret_cast<const float *>(base + (size_t)(3 + a) * kRow);
      const float q_hi = (float)inv_1m[a];
      sa.co = LineCoef<float>{pf, (float)lam[a], (float)scale, q_hi, pf + kRow, (float)(inv_1m[a] - (double)q_hi),
                              1.0 - 1.0 / inv_1m[a] > 0x1p-24 ? 1 : 0};
      e = launch_sweep<float>(a, PRO_LOAD, EPI_STORE, 1, sa, s);
    } else {
      SweepArgs<double> sa;
      memset(&sa, 0, sizeof(sa));
      sa.f[0] = (double *)psi;
      sa.fin[0] = a == 0 ? (const double *)f : nullptr;
      for (int q = 0; q < 3; ++q) sa.n[q] = q < dim ? n[q] : 1;
      sa.dim = dim;
      sa.co = LineCoef<double>{base + (size_t)a * kRow, lam[a], scale, inv_1m[a], nullptr, 0.0, 0};
      e = launch_sweep<double>(a, PRO_LOAD, EPI_STORE, 1, sa, s);
    }
    if (e != cudaSuccess) return ib_internal_fail(IB_ERR_CUDA, cudaGetErrorString(e));
  }
  return IB_OK;
}
