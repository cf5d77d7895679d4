// Internal declarations of the sm_103a IB-GM implementation (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ibg {

// Coefficients of one constant-coefficient cyclic line operator
//   A = (1 + 2r) I - r (S + S^{-1})      (S the cyclic shift, eq. TriDiagX)
// written as the exact product A = c (I - lam S)(I - lam S^{-1}) with
// lam = 2r / (1 + 2r + sqrt(1 + 4r)) in [0, 1) and c = r / lam.  The inverse is
// two first-order cyclic recurrences and a scale; each recurrence is a
// non-periodic pass plus a rank-one periodic correction with weight
// 1 / (1 - lam^n).
template <typename T>
struct LineCoef {
  const T *pw;  // lam^k for k = 0 .. n  (device)
  T lam;
  T inv_c;      // 1 / c
  T inv_1m;     // 1 / (1 - lam^n)
};

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
  T inv_h[3];
  int n[3];
  int dim;
  LineCoef<T> co;
};

template <typename T>
struct RhsArgs {
  const T *u[3];
  const T *p, *psi;
  T *Nold[3];     // in: N(u^{n-1}); out: N(u^n)
  T *scr[3];      // in: spread force f; out: R = u* - u^n
  T inv_h[3], inv_h2[3];
  T mu, inv_rho, dt;
  int n[3];
  int first;      // n == 0: p* = 0 and N^{1/2} = N(u^0)
};

struct MarkerArgs {
  // markers, FP64 SoA
  double *X[3];   // X^n (updated to X^{n+1} by the force kernel)
  double *Xh[3];  // X^{n+1/2}
  double *U[3];   // U^n
  double *Uold[3];// U^{n-1}
  double *G[3];   // nodal force at X^{n+1/2}
  const int64_t *row;   // CSR over markers: neighbours of marker a are
  const int32_t *col;   //   col[row[a] .. row[a+1]) with
  const double *kap;    //   spring constants kap[] and rest lengths rest[]
  const double *rest;
  int64_t nm;
  double dt, H;
  double inv_h[3];
  double inv_vol;       // 1 / h^d
  int n[3];
  int dim, kernel, first;
};

// launchers (return cudaError_t of the launch)
template <typename T>
cudaError_t launch_sweep(int axis, int pro, int epi, int nfields, const SweepArgs<T> &a, cudaStream_t s);
template <typename T>
cudaError_t launch_rhs(int dim, const RhsArgs<T> &a, cudaStream_t s);
template <typename T>
cudaError_t launch_divergence(int dim, const T *const u[3], T *div, const int n[3], const T inv_h[3],
                              cudaStream_t s);
template <typename T>
cudaError_t launch_interp(const MarkerArgs &m, const T *const u[3], cudaStream_t s);
cudaError_t launch_force(const MarkerArgs &m, cudaStream_t s);
template <typename T>
cudaError_t launch_spread(const MarkerArgs &m, T *const f[3], cudaStream_t s);

cudaError_t launch_markers_layout(double *aos, double *const X[3], int64_t nm, int dim, int to_soa,
                                  cudaStream_t s);

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
