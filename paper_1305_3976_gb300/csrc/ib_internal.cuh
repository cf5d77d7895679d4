// Internal declarations of the sm_103a IB-GM implementation (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ibg {

// Programmatic dependent launch.  The step's kernels are launched with
// launch_pdl, so a kernel's CTAs can be scheduled while the previous kernel of
// the stream drains; every such kernel calls pdl_wait() before its first
// global memory access (it returns once the previous kernel has completed and
// its writes are visible; without the launch attribute it returns at once)
// and pdl_release() to let the next kernel be scheduled early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// SM count of the current device (0 if the query fails), for grids sized in
// multiples of it
inline long long device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return sms;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Block coordinates of a kernel body.  An ordinary launch passes the hardware
// blockIdx / gridDim (hw_blk); a batched launch -- the grids of one ensemble
// size class stepped by a single launch -- passes each member's own block
// index and grid inside its share of the launch (batch_member).
struct Blk {
  unsigned x, y, z;     // block index
  unsigned gx, gy, gz;  // grid size
};
__device__ __forceinline__ Blk hw_blk() { return Blk{blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y, gridDim.z}; }

// Arguments of a batched launch, passed by value as one kernel parameter
// (constant bank): per member its arguments and its own 3-D grid; the
// launch's 1-D grid is the concatenation of the members' grids.
constexpr int kBatch = 24;
template <typename A>
struct Batch {
  A a[kBatch];
  unsigned start[kBatch + 1];  // first block of member m; start[n] = blocks of the launch
  unsigned gx[kBatch], gy[kBatch];
  int n;
};

// the member that owns this block and the block's coordinates in its grid
template <typename A>
__device__ __forceinline__ int batch_member(const Batch<A> &B, Blk &b) {
  const unsigned v = blockIdx.x;
  int m = 0;
  while (m + 1 < B.n && v >= B.start[m + 1]) ++m;
  const unsigned l = v - B.start[m], gx = B.gx[m], gy = B.gy[m];
  b.x = l % gx;
  b.y = (l / gx) % gy;
  b.z = l / (gx * gy);
  b.gx = gx;
  b.gy = gy;
  b.gz = (B.start[m + 1] - B.start[m]) / (gx * gy);
  return m;
}

// Launch `kernel` over n members (args[i] with grid grids[i]), kBatch members
// per launch, with smem bytes of dynamic shared memory per CTA; `extra`
// follows the batch in the kernel's parameters.
template <typename A, typename K, typename... Extra>
cudaError_t launch_batch_smem(K kernel, const A *args, const dim3 *grids, int n, dim3 block, size_t smem,
                              cudaStream_t s, Extra... extra) {
  for (int c0 = 0; c0 < n; c0 += kBatch) {
    Batch<A> B;
    const int k = n - c0 < kBatch ? n - c0 : kBatch;
    unsigned tot = 0;
    for (int i = 0; i < kBatch; ++i) {
      if (i < k) {
        B.a[i] = args[c0 + i];
        B.gx[i] = grids[c0 + i].x;
        B.gy[i] = grids[c0 + i].y;
      } else {
        B.a[i] = args[c0];
        B.gx[i] = B.gy[i] = 1;
      }
      B.start[i] = tot;
      if (i < k) tot += grids[c0 + i].x * grids[c0 + i].y * grids[c0 + i].z;
    }
    B.start[kBatch] = tot;
    B.n = k;
    if (tot == 0) continue;
    cudaError_t e = launch_pdl(kernel, dim3(tot), block, smem, s, B, extra...);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
template <typename A, typename K, typename... Extra>
cudaError_t launch_batch(K kernel, const A *args, const dim3 *grids, int n, dim3 block, cudaStream_t s,
                         Extra... extra) {
  return launch_batch_smem(kernel, args, grids, n, block, 0, s, extra...);
}

// 4 contiguous elements at p (16-byte aligned for float, 32 for double)
__device__ __forceinline__ void ld4(const float *p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4 *>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&v)[4]) {
  const double2 a = reinterpret_cast<const double2 *>(p)[0];
  const double2 b = reinterpret_cast<const double2 *>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float *p, const float (&v)[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double *p, const double (&v)[4]) {
  reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}


// Coefficients of one constant-coefficient cyclic line operator
//   A = (1 + 2r) I - r (S + S^{-1})      (S the cyclic shift, eq. TriDiagX)
// written as the exact product A = c (I - lam S)(I - lam S^{-1}) with
// lam = 2r / (1 + 2r + sqrt(1 + 4r)) in [0, 1) and c = r / lam.  The inverse is
// two first-order cyclic recurrences and a scale; each recurrence is a
// non-periodic pass plus a rank-one periodic correction with weight
// 1 / (1 - lam^n).  The scale is applied once, in the sweep's epilogue: a
// chain of sweeps (each one linear) passes 1 in all sweeps but the last,
// which carries the product of the chain's 1/c.
//
// The periodic correction of each factor -- the rank-one term
// lam^{i+1} z_{n-1} / (1 - lam^n) (Sherman-Morrison on the factor), combined
// with a chunk's carry-in c as t = lam^{i0} K + c, K = z_{n-1} / (1 - lam^n)
// -- is evaluated to FP64 accuracy when wrap_ext is set (FP32 fields whose
// wrap weight lam^n is above FP32 resolution, e.g. the psi operator with
// r = 1/h^2, where lam^n is about e^-1): the FP64 host values of lam^{i0} and
// 1/(1 - lam^n) are split into FP32 pairs hi + lo, and the product and sum
// are carried in two-float arithmetic (wrap_term_ext), so t is rounded to FP32
// once.  FP64 instructions would do the same at 1/64 of the FP32 rate on this
// GPU's FP64 pipe.
template <typename T>
struct LineCoef {
  const T *pw;     // lam^k for k = 0 .. n  (device)
  T lam;
  T scale;         // factor applied to the solution: 1 / c for one complete solve
  T inv_1m;        // 1 / (1 - lam^n)
  const T *pw_lo;  // FP32: lam^k - pw[k] in FP32 (device; read when wrap_ext)
  T inv_1m_lo;     // FP32: 1 / (1 - lam^n) - inv_1m
  int wrap_ext;    // FP64-accurate periodic correction (T = float only)
};

// t = (p_hi + p_lo) tot (q_hi + q_lo) + cin in two-float arithmetic: the
// rounding error of each product comes exactly from an FMA and that of the
// final sum from Knuth's two-sum, so about 46 significant bits reach the one
// rounding to FP32.  The expressions are evaluated in source order (no
// reassociation without fast-math flags).
__device__ __forceinline__ float wrap_term_ext(float p_hi, float p_lo, float q_hi, float q_lo, float tot, float cin) {
  const float k_hi = tot * q_hi;
  const float k_lo = fmaf(tot, q_lo, fmaf(tot, q_hi, -k_hi));
  const float m_hi = p_hi * k_hi;
  const float m_lo = fmaf(p_hi, k_lo, fmaf(p_lo, k_hi, fmaf(p_hi, k_hi, -m_hi)));
  const float s = m_hi + cin;
  const float bb = s - m_hi;
  const float e = (m_hi - (s - bb)) + (cin - bb);
  return s + (e + m_lo);
}
__device__ __forceinline__ double wrap_term_ext(double, double, double, double, double tot, double cin) {
  return tot + cin;  // not used: FP64 fields take the plain correction
}

// t = lam^{i0} tot / (1 - lam^n) + cin for a chunk starting at element i0 of
// a line whose non-periodic end value (the factor's carry over all chunks) is
// tot
// tot (EXT: to FP64 accuracy; the kernels are instantiated with EXT for the
// FP32 solves whose LineCoef::wrap_ext is set)
template <bool EXT, typename T>
__device__ __forceinline__ T wrap_term(const LineCoef<T> &co, int i0, T tot, T cin) {
  if (EXT) return wrap_term_ext(__ldg(co.pw + i0), __ldg(co.pw_lo + i0), co.inv_1m, co.inv_1m_lo, tot, cin);
  return fma(__ldg(co.pw + i0), tot * co.inv_1m, cin);
}

enum { PRO_LOAD = 0, PRO_DIV = 1 };
enum { EPI_STORE = 0, EPI_ADDU = 1, EPI_P = 2 };

template <typename T>
struct SweepArgs {
  T *f[3];        // fields solved (in place unless fin is set), one per blockIdx.y/z
  const T *fin[3];// PRO_LOAD: right-hand sides read from here instead of f (may be null)
  const T *u[3];  // PRO_DIV: velocity u^{n+1}
  T *uo[3];       // EPI_ADDU: u^n, receives u^n + e
  T *p;           // PRO_DIV / EPI_P: pressure
  T *div;         // PRO_DIV: D.u^n in, D.u^{n+1} out
  T pro_scale;    // PRO_DIV: -rho / dt
  T chi_mu_half;  // PRO_DIV: chi mu / 2
  T p_keep;       // PRO_DIV: weight of p^{n-1/2} in p^{n+1/2} (1; 0 in the first-order variant)
  T inv_h[3];
  int n[3];
  int dim;
  LineCoef<T> co;
};

template <typename T>
struct RhsArgs {
  const T *u[3];
  const T *p, *psi;  // p* = p + psi (psi null: p* = p, the first-order variant)
  T *Nold[3];     // in: N(u^{n-1}); out: N(u^n)
  T *scr[3];      // out: R = u* - u^n without the force term (spreading adds dt/rho f)
  T inv_h[3], inv_h2[3];
  // R = cmu L u + ncg_c (p* - p*(-c)) + ncA N^n + cN N^{n-1} with the
  // Laplacian L u = sum_a (u(+a) + u(-a)) / h_a^2 - 2 u sum_a 1 / h_a^2
  // (its coefficients cancel exactly on a constant field)
  T cmu;          // dt mu / rho
  T ncg[3];       // -dt / (rho h_a)
  T ncA, cN;      // -3/2 dt and 1/2 dt (n == 0: -dt and 0)
  int n[3];
  int first;      // n == 0: p* = 0 and N^{1/2} = N(u^0)
};

struct MarkerArgs {
  double *X[3];     // X^n, FP64 (advanced to X^{n+1} by the update kernel)
  double *Xh[3];    // X^{n+1/2}, FP64
  void *U[3];       // U^n, field precision
  void *Uold[3];    // U^{n-1}, field precision
  void *G[3];       // nodal force at X^{n+1/2}, field precision
  // grid locations, slot 2a + o for axis a and MAC offset o (0: own axis,
  // 1: half a cell): index of the first stencil node (in [0, n_a)) and the 4
  // node weights
  int32_t *locI_b;  // [2d][nm] of X^n (interpolation)
  void *locI_w;     // [2d][nm][4] field precision
  int32_t *locS_b;  // [2d][nm] of X^{n+1/2} (spreading)
  void *locS_w;
  void *locS_f;     // [d][nm] field precision: fraction of X^{n+1/2} / h on the own-axis offset
  const int64_t *row;   // CSR over markers: neighbours of marker a are
  const int32_t *col;   //   col[row[a] .. row[a+1]) with
  const double *kap;    //   spring constants kap[] and rest lengths rest[]
  const double *rest;
  const void *kapT, *restT;  // the same in the field precision
  int64_t nm;
  double dt, H;
  double inv_h[3];
  double spread_scale;  // dt / (rho h^d): spreading adds dt/rho f to R
  float h32[3], inv_n32[3];  // h_a and 1 / n_a for the location-based force
  int n[3];
  int dim, kernel, first;
  int frac_force;       // force from the stored locations of X^{n+1/2} (FP32 fields)
};

// marker arguments with three field pointers: the velocity interpolation
// reads (const) or the momentum increments spreading adds to
struct MarkerFieldArgs {
  MarkerArgs m;
  void *f[3];
};

// strided line solves staged by TMA (see ib_sweep_tma.cu): FP32, y and z
// lines, plain load/store sweeps; autotuner candidate id kTmaCfg
constexpr int kTmaCfg = 11;
struct SweepTmaMaps {
  CUtensorMap in[3], out[3];  // per field: boxes of 32 x columns x (part of) a line
  int nfields;
};
bool sweep_tma_ok(const SweepArgs<float> &a, int axis);
void sweep_tma_shape(int nl, int *ch, int *w);
cudaError_t launch_sweep_tma(int axis, int nfields, const SweepArgs<float> &a, cudaStream_t s);
// process-wide flag set by a kernel whose bounded wait ran out; returns its
// value and clears it
int take_wait_timeout();
// a kernel whose mbarrier wait cannot complete and runs out after limit_ns
cudaError_t launch_wait_selftest(unsigned long long limit_ns, cudaStream_t s);

// adjoint step (see ib_adjoint.cu)
template <typename T>
struct AdjFields {
  T *ub[3], *pb, *psib, *nbar[3], *divb;  // bars of u, p, psi, N(u^{n-1}), D.u
  T *q, *rb[3], *vv[3];                   // temporaries
  long long cells;
  int n[3];
  int dim;
  T ih[3];
  T chi_mu_half, rho_dt, dt_mu_rho, dt_rho, dt;
  T p_keep;  // weight of p^{n-1/2} in p^{n+1/2}
  T psi_w;   // weight of psi^{n-1/2} in p*
};

template <typename T>
struct AdjMarkers {
  const double *X[3];  // X^n (from the tape)
  const T *Uold[3];    // U^{n-1} (from the tape)
  T *U[3];             // U^n (recomputed)
  double *Xh[3];       // X^{n+1/2} (recomputed)
  T *G[3];             // nodal force (recomputed)
  T *Gb[3];            // bars of G, X^{n+1/2}, X, U, U^{n-1}
  double *Xhb[3];
  double *Xb[3];
  T *Ub[3];
  T *Uoldb[3];
  const int64_t *row;
  const int32_t *col;
  const double *kap;
  const int32_t *cedge;  // connection index of every CSR entry
  double *dk;            // d(loss)/d kappa, per connection
  // stencils of X^n (set 0) and X^{n+1/2} (set 1) for every (marker,
  // component) pair p = k d + c: first node per axis stb[a np + p], node
  // weights stw[(4 a + j) np + p] and their derivatives stdw (same layout)
  int32_t *stb[2];
  T *stw[2], *stdw[2];
  int64_t nm;
  double dt, H;
  double inv_h[3];
  double inv_vol;
  int n[3];
  int dim, kernel, first;
};

template <typename T>
cudaError_t adjoint_fields_a(const AdjFields<T> &f, cudaStream_t s);
template <typename T>
cudaError_t adjoint_fields_b(const AdjFields<T> &f, cudaStream_t s);
template <typename T>
cudaError_t adjoint_fields_c(const AdjFields<T> &f, const T *const u[3], int first, cudaStream_t s);
template <typename T>
cudaError_t adjoint_markers_pre(const AdjMarkers<T> &am, const T *const u[3], cudaStream_t s);
template <typename T>
cudaError_t adjoint_markers_post(const AdjMarkers<T> &am, const T *const rb[3], T dt_rho, const T *const u[3],
                                 T *const ub[3], cudaStream_t s);

// launchers (return cudaError_t of the launch)
template <typename T>
cudaError_t launch_sweep(int axis, int pro, int epi, int nfields, const SweepArgs<T> &a, cudaStream_t s,
                         int cfg = -1);
int sweep_candidates(int axis, int nl, int nx, bool dbl, int *out, int max);
void sweep_config_shape(int axis, int cfg, int nl, int *a, int *b, int *c);
template <typename T>
cudaError_t launch_rhs(int dim, const RhsArgs<T> &a, cudaStream_t s);
template <typename T>
cudaError_t launch_divergence(int dim, const T *const u[3], T *div, const int n[3], const T inv_h[3],
                              cudaStream_t s);
template <typename T>
cudaError_t launch_locate(const MarkerArgs &m, cudaStream_t s);
template <typename T>
cudaError_t launch_interp(const MarkerArgs &m, const T *const u[3], cudaStream_t s);
template <typename T>
cudaError_t launch_update(const MarkerArgs &m, cudaStream_t s);
template <typename T>
cudaError_t launch_force(const MarkerArgs &m, cudaStream_t s);
template <typename T>
cudaError_t launch_spread(const MarkerArgs &m, T *const f[3], cudaStream_t s);

cudaError_t launch_markers_layout(double *aos, double *const X[3], const int32_t *perm, int64_t nm, int dim,
                                  int to_soa, cudaStream_t s);

// batched launches over n grids of one ensemble size class (same dim and
// precision; see launch_batch)
template <typename T>
cudaError_t launch_interp_batch(const MarkerFieldArgs *a, int n, cudaStream_t s);
template <typename T>
cudaError_t launch_update_batch(const MarkerArgs *m, int n, cudaStream_t s);
template <typename T>
cudaError_t launch_force_batch(const MarkerArgs *m, int n, cudaStream_t s);
template <typename T>
cudaError_t launch_spread_batch(const MarkerFieldArgs *a, int n, cudaStream_t s);
template <typename T>
cudaError_t launch_rhs_batch(int dim, const RhsArgs<T> *a, int n, cudaStream_t s);
template <typename T>
cudaError_t launch_sweep_batch(int axis, int pro, int epi, int nfields, const SweepArgs<T> *a, int n,
                               cudaStream_t s, int cfg);
// the FP32 sweeps with the FP64-accurate periodic correction (LineCoef::wrap_ext)
cudaError_t launch_sweep_f32_ext(int axis, int pro, int epi, int nfields, const SweepArgs<float> &a, cudaStream_t s,
                                 int cfg);
cudaError_t launch_sweep_batch_f32_ext(int axis, int pro, int epi, int nfields, const SweepArgs<float> *a, int n,
                                       cudaStream_t s, int cfg);

struct DiagAccum {
  double div2, divmax, kin, vol, elastic, nonfinite;
};
template <typename T>
cudaError_t launch_field_diag(int dim, const T *const u[3], const T *p, const T *div, const int n[3],
                              double *acc, cudaStream_t s);
cudaError_t launch_marker_diag(int dim, const double *const X[3], int64_t nm, const int32_t *edges,
                               const double *kappa, const double *rest, int64_t ne, const int32_t *tris,
                               int64_t nt, double H, double *acc, cudaStream_t s);

}  // namespace ibg
