// Discrete adjoint of one IB-GM step (Sec. 3.4, Steps 1a-3f) for sm_103a.
//
// The step maps the state S^n = (u, p, psi, N(u^{n-1}), D.u, X, U^{n-1}) to
// S^{n+1}; with connection stiffnesses kappa as parameters.  Given the
// adjoint (bar) of S^{n+1}, the kernels below produce the bar of S^n and add
// d(loss)/d kappa.  Structure, in reverse order of the forward step:
//   3f/3e  p' = p - chi mu/2 (D.u' + D.u) + psi',  psi' = A^{-1}(-rho/dt D.u')
//          (first-order variant of Sec. 3.1: p' = psi', and p* = p below)
//          with A = prod (I - D_aa) symmetric, and D^T = -G;
//   3c-3d  u' = u + M^{-1} R, M = prod (I - a D_aa) symmetric;
//   3a-3b  R = dt [(mu L u - G p* + f)/rho - (c1 N(u) + c2 N(u^{n-1}))],
//          N quadratic in u (its Jacobian-transpose gathered per target face);
//   2b     f = S(X^{n+1/2}) G (spreading; adjoint: interpolation, plus the
//          derivative of the weights),
//   2a     G = F(X^{n+1/2}; kappa), zero rest length: G_a = sum kappa (X_b - X_a),
//   1b-1c  X' = X + dt V, X^{n+1/2} = X + dt V / 2, V = c1 U + c2 U^{n-1},
//   1a     U = J(X) u (interpolation; adjoint: spreading, plus the derivative
//          of the weights).
// (c1, c2) = (3/2, -1/2), or (1, 0) on the first step.
#include <math.h>

#include "ib_internal.cuh"

namespace ibg {

namespace {

__device__ __forceinline__ float sinpi_t(float x) { return sinpif(x); }
__device__ __forceinline__ double sinpi_t(double x) { return sinpi(x); }
__device__ __forceinline__ float cospi_a(float x) { return cospif(x); }
__device__ __forceinline__ double cospi_a(double x) { return cospi(x); }

__device__ __forceinline__ int wrapi(int i, int n) {
  if (i >= 0 && i < n) return i;
  int r = i % n;
  return r < 0 ? r + n : r;
}

// weights of the 4 stencil nodes and their derivatives with respect to the
// fraction f (see the forward kernels for the closed form)
template <typename T>
__device__ __forceinline__ void weights_d(T f, int kernel, T (&w)[4], T (&dw)[4]) {
  if (kernel == 0) {
    const T q = sqrt(T(1) + T(4) * f * (T(1) - f));
    const T dq = (T(2) - T(4) * f) / q;
    const T a = T(3) - T(2) * f, b = T(1) + T(2) * f;
    w[0] = (a - q) * T(0.125);
    w[1] = (a + q) * T(0.125);
    w[2] = (b + q) * T(0.125);
    w[3] = (b - q) * T(0.125);
    dw[0] = (T(-2) - dq) * T(0.125);
    dw[1] = (T(-2) + dq) * T(0.125);
    dw[2] = (T(2) + dq) * T(0.125);
    dw[3] = (T(2) - dq) * T(0.125);
  } else {
    const T pi_8 = T(0.39269908169872415);  // pi / 8
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const T r = (T(j - 1) - f) * T(0.5);
      w[j] = T(0.25) * (T(1) + cospi_a(r));
      dw[j] = pi_8 * sinpi_t(r);
    }
  }
}

// stencil of component c at position X (FP64): first node per axis, weights
// and their derivatives with respect to X_a (d/dX = d/df / h)
template <typename T, int DIM>
__device__ __forceinline__ void stencil_at(const double *const *X, long long k, int c, const double *inv_h,
                                           int kernel, int (&b)[3], T (&w)[3][4], T (&dw)[3][4]) {
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const double x = X[a][k] * inv_h[a] - (a == c ? 0.0 : 0.5);
    const double fl = floor(x);
    const T f = (T)(x - fl);
    b[a] = (int)fl - 1;
    weights_d<T>(f, kernel, w[a], dw[a]);
#pragma unroll
    for (int j = 0; j < 4; ++j) dw[a][j] *= (T)inv_h[a];
  }
}

}  // namespace

// A1: q = psi_bar + p_bar
template <typename T>
__global__ void k_adj_q(const T *psib, const T *pb, T *q, long long cells) {
  for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < cells; o += (long long)gridDim.x * blockDim.x)
    q[o] = psib[o] + pb[o];
}

// A3: with q = A^{-1}(psi_bar + p_bar):  D.u' bar  = divb - chi mu/2 pb - rho/dt q
// (stored in q); the bar of D.u^n is -chi mu/2 pb
// (first-order variant: chi = 0 and p' = psi', so the bar of p^n keeps
// p_keep = 0 of pb)
template <typename T>
__global__ void k_adj_div(T *q, T *divb, T *pb, T chi_mu_half, T rho_dt, T p_keep, long long cells) {
  for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < cells; o += (long long)gridDim.x * blockDim.x) {
    const T p = pb[o];
    q[o] = divb[o] - chi_mu_half * p - rho_dt * q[o];
    divb[o] = -chi_mu_half * p;
    pb[o] = p_keep * p;
  }
}

// A4: u' bar (total) = ub - G(D.u' bar); also copied to Rb for the solves
// (one thread per x index, blockIdx.y / z the other coordinates)
template <typename T, int DIM>
__global__ void __launch_bounds__(128) k_adj_grad(T *ub0, T *ub1, T *ub2, T *rb0, T *rb1, T *rb2, const T *q, int nx,
                                                  int ny, int nz, T ihx, T ihy, T ihz) {
  T *ub[3] = {ub0, ub1, ub2}, *rb[3] = {rb0, rb1, rb2};
  const T ih[3] = {ihx, ihy, ihz};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nx) {
    const int j = blockIdx.y, k = blockIdx.z;
    const int o = i + nx * (j + ny * k);
    const int dm[3] = {i == 0 ? nx - 1 : -1, j == 0 ? nx * (ny - 1) : -nx, k == 0 ? nx * ny * (nz - 1) : -nx * ny};
    const T q0 = q[o];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const T v = ub[c][o] - (q0 - q[o + dm[c]]) * ih[c];
      ub[c][o] = v;
      rb[c][o] = v;
    }
  }
}

// A5 (after the momentum solves Rb = M^{-1} u'bar):
//   ub += dt mu/rho L Rb;  (n > 0) pb += dt/rho D.Rb, psib = psi_w dt/rho D.Rb;
//   V = -dt c1 Rb + Nb (the bar of N(u^n), scattered by k_adj_adv);
//   Nb = -c2 (-dt) Rb ... = dt/2 Rb (n > 0) or 0
// One thread per x index, blockIdx.y / z the other coordinates (32-bit
// offsets: fields hold fewer than 2^31 elements).
template <typename T, int DIM>
__global__ void __launch_bounds__(128) k_adj_rhs(T *ub0, T *ub1, T *ub2, const T *rb0, const T *rb1, const T *rb2,
                                                 T *nb0, T *nb1, T *nb2, T *v0, T *v1, T *v2, T *pb, T *psib, int nx,
                                                 int ny, int nz, T ihx, T ihy, T ihz, T dt_mu_rho, T dt_rho, T dt,
                                                 T psi_w, int first) {
  T *ub[3] = {ub0, ub1, ub2}, *nb[3] = {nb0, nb1, nb2}, *vv[3] = {v0, v1, v2};
  const T *rb[3] = {rb0, rb1, rb2};
  const T ih[3] = {ihx, ihy, ihz};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nx) {
    const int j = blockIdx.y, k = blockIdx.z;
    const int o = i + nx * (j + ny * k);
    const int dp[3] = {i + 1 == nx ? 1 - nx : 1, j + 1 == ny ? nx * (1 - ny) : nx,
                       k + 1 == nz ? nx * ny * (1 - nz) : nx * ny};
    const int dm[3] = {i == 0 ? nx - 1 : -1, j == 0 ? nx * (ny - 1) : -nx, k == 0 ? nx * ny * (nz - 1) : -nx * ny};
    T divR = T(0);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const T r0 = rb[c][o];
      T lap = T(0);
#pragma unroll
      for (int a = 0; a < DIM; ++a) lap += (rb[c][o + dp[a]] - T(2) * r0 + rb[c][o + dm[a]]) * ih[a] * ih[a];
      ub[c][o] += dt_mu_rho * lap;
      divR += (rb[c][o + dp[c]] - r0) * ih[c];
      const T c1 = first ? T(1) : T(1.5);
      vv[c][o] = -dt * c1 * r0 + nb[c][o];
      nb[c][o] = first ? T(0) : T(0.5) * dt * r0;
    }
    if (!first) {
      pb[o] += dt_rho * divR;
      psib[o] = psi_w * dt_rho * divR;
    } else {
      psib[o] = T(0);
    }
  }
}

// A6: ub += (dN/du)^T V with N the skew-symmetric advection of the forward
// step.  For component c and axis a the forward term at face x is
//   1/2 (A+(x) u_c(x+a) - A-(x) u_c(x-a)) / h_a,
// a == c: A+ = (u_c(x) + u_c(x+a))/2, A- = (u_c(x-a) + u_c(x))/2;
// a != c: A+ = (u_a(x+a) + u_a(x+a-c))/2, A- = (u_a(x) + u_a(x-c))/2.
// With S_ca(x) = V_c(x) / (2 h_a) its transpose scatters, per source x,
//   a == c: S (u_c(x+a) - u_c(x-a))/2 to u_c(x), S (u_c(x+a)/2 + A+) to
//           u_c(x+a), -S (u_c(x-a)/2 + A-) to u_c(x-a);
//   a != c: S u_c(x+a)/2 to u_a(x+a) and u_a(x+a-c), S A+ to u_c(x+a),
//           -S u_c(x-a)/2 to u_a(x) and u_a(x-c), -S A- to u_c(x-a).
// The kernel gathers instead: the thread of face y of component b sums every
// term whose target is (b, y), reading V and u around y, and adds the sum to
// ub_b(y) once (no atomics, a fixed summation order).
// One thread per face x index, blockIdx.y / z the other two coordinates;
// neighbour offsets along each axis are periodic 32-bit steps (fields hold
// fewer than 2^31 elements), combined additively across axes.
template <typename T, int DIM>
__global__ void __launch_bounds__(128) k_adj_adv(T *ub0, T *ub1, T *ub2, const T *u0, const T *u1, const T *u2,
                                                 const T *v0, const T *v1, const T *v2, int nx, int ny, int nz,
                                                 T ihx, T ihy, T ihz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
  const int j = blockIdx.y, k = blockIdx.z;
  const int o = i + nx * (j + ny * k);
  T *ub[3] = {ub0, ub1, ub2};
  const T *u[3] = {u0, u1, u2}, *vv[3] = {v0, v1, v2};
  const T ih[3] = {ihx, ihy, ihz};
  // offsets of y + e_a (pl) and y - e_a (mi)
  const int pl[3] = {i + 1 == nx ? 1 - nx : 1, j + 1 == ny ? nx * (1 - ny) : nx,
                     DIM == 3 ? (k + 1 == nz ? nx * ny * (1 - nz) : nx * ny) : 0};
  const int mi[3] = {i == 0 ? nx - 1 : -1, j == 0 ? nx * (ny - 1) : -nx,
                     DIM == 3 ? (k == 0 ? nx * ny * (nz - 1) : -nx * ny) : 0};
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    const T *vb = vv[b], *ubv = u[b];
    T acc = T(0);
    const int ymb = o + mi[b];  // y - b
    // a == c == b: sources y, y - b, y + b
    {
      const int yp = o + pl[b], ym = ymb;
      const T uy = ubv[o], up = ubv[yp], um = ubv[ym];
      const T sy = T(0.5) * ih[b] * vb[o], sm = T(0.5) * ih[b] * vb[ym], sp = T(0.5) * ih[b] * vb[yp];
      acc += sy * (T(0.5) * up - T(0.5) * um);
      acc += sm * (T(0.5) * uy + T(0.5) * (um + uy));
      acc -= sp * (T(0.5) * uy + T(0.5) * (uy + up));
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      if (a == b) continue;
      // c = b, axis a: S_ba A+ from source y - a, -S_ba A- from source y + a
      const int ya_m = o + mi[a], ya_p = o + pl[a], yab = o + pl[a] + mi[b];  // y - a, y + a, y + a - b
      const T *ua = u[a];
      const T Ap = T(0.5) * (ua[o] + ua[ymb]);
      const T Am = T(0.5) * (ua[ya_p] + ua[yab]);
      acc += T(0.5) * ih[a] * vb[ya_m] * Ap;
      acc -= T(0.5) * ih[a] * vb[ya_p] * Am;
      // c = a != b, axis b: the terms of component a's advection along b
      // whose targets are u_b: S_ab u_a / 2 from sources y - b and
      // y - b + a, -S_ab u_a / 2 from sources y and y + a
      const T *va = vv[a];
      const T shb = T(0.5) * ih[b];
      acc += shb * va[ymb] * T(0.5) * ua[o];
      acc += shb * va[yab] * T(0.5) * ua[ya_p];
      acc -= shb * va[o] * T(0.5) * ua[ymb];
      acc -= shb * va[ya_p] * T(0.5) * ua[yab];
    }
    ub[b][o] += acc;
  }
}

// --------------------------------------------------------------------------
// markers.  The FP64 position arithmetic of a stencil (first node, weights
// and their derivatives) runs once per (marker, component) pair in
// k_adj_stencil, one pair per thread (GB300's FP64 pipe issues a warp
// instruction at the same cost for 1 or 32 lanes); the node work then runs in
// groups of ROWS lanes per pair (16 in 3D, 4 in 2D), lane r owning the stencil
// row (y, z) = (r & 3, r >> 2), with shuffle reductions over the group.

// stencil of every pair at the positions X (set 0: X^n, set 1: X^{n+1/2})
template <typename T, int DIM>
__global__ void k_adj_stencil(AdjMarkers<T> am, int set) {
  const long long np = am.nm * DIM;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const long long k = p / DIM;
  const int c = (int)(p % DIM);
  int b[3];
  T w[3][4], dw[3][4];
  stencil_at<T, DIM>(set ? (const double *const *)am.Xh : am.X, k, c, am.inv_h, am.kernel, b, w, dw);
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    am.stb[set][a * np + p] = b[a];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      am.stw[set][(4 * a + j) * np + p] = w[a][j];
      am.stdw[set][(4 * a + j) * np + p] = dw[a][j];
    }
  }
}

// the lane's pair, its stencil row and the row's 4 node offsets
template <typename T, int DIM>
struct AdjRow {
  static constexpr int ROWS = DIM == 3 ? 16 : 4;
  long long p, k;
  int c, jy, kz;
  bool valid;
  T wx[4], dwx[4], wy, dwy, wz, dwz;
  long long node[4];
  __device__ __forceinline__ AdjRow(const AdjMarkers<T> &am, int set) {
    const long long np = am.nm * DIM;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    p = t / ROWS;
    const int r = (int)(t % ROWS);
    jy = r & 3;
    kz = DIM == 3 ? r >> 2 : 0;
    valid = p < np;
    k = valid ? p / DIM : 0;
    c = valid ? (int)(p % DIM) : 0;
    wy = dwy = dwz = T(0);
    wz = T(1);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      wx[j] = dwx[j] = T(0);
      node[j] = 0;
    }
    if (!valid) return;
    const int32_t *sb = am.stb[set];
    const T *sw = am.stw[set], *sdw = am.stdw[set];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      wx[j] = sw[j * np + p];
      dwx[j] = sdw[j * np + p];
    }
    wy = sw[(4 + jy) * np + p];
    dwy = sdw[(4 + jy) * np + p];
    if (DIM == 3) {
      wz = sw[(8 + kz) * np + p];
      dwz = sdw[(8 + kz) * np + p];
    }
    const int bx = sb[p];
    const long long row = (long long)am.n[0] * (wrapi(sb[np + p] + jy, am.n[1]) +
                                                (DIM == 3 ? (long long)am.n[1] * wrapi(sb[2 * np + p] + kz, am.n[2]) : 0));
#pragma unroll
    for (int j = 0; j < 4; ++j) node[j] = row + wrapi(bx + j, am.n[0]);
  }
};

template <int ROWS, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int off = ROWS / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// 1a: U_c = J(X^n) u_c
template <typename T, int DIM>
__global__ void k_adj_interp_fwd(AdjMarkers<T> am, const T *u0, const T *u1, const T *u2) {
  AdjRow<T, DIM> L(am, 0);
  T s = T(0);
  if (L.valid) {
    const T *uc = L.c == 0 ? u0 : (L.c == 1 ? u1 : u2);
#pragma unroll
    for (int j = 0; j < 4; ++j) s += uc[L.node[j]] * L.wx[j];
    s *= L.wy * L.wz;
  }
  s = group_sum<AdjRow<T, DIM>::ROWS>(s);
  if (L.valid && L.jy == 0 && L.kz == 0) am.U[L.c][L.k] = s;
}

// 1b-1c: X^{n+1/2} = X + dt V / 2
template <typename T, int DIM>
__global__ void k_adj_half(AdjMarkers<T> am) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= am.nm * DIM) return;
  const long long k = t / DIM;
  const int c = (int)(t % DIM);
  const double U = (double)am.U[c][k];
  const double vel = am.first ? U : 1.5 * U - 0.5 * (double)am.Uold[c][k];
  const double Xc = am.X[c][k];
  am.Xh[c][k] = 0.5 * ((Xc + am.dt * vel) + Xc);
}

// 2b adjoint: Gb_c = sum_nodes fb_c W / h^d  (fb = dt/rho Rb); and the
// derivative of the weights: Xhb_a += G_c sum_nodes fb_c dW/dX_a / h^d
template <typename T, int DIM>
__global__ void k_adj_spread_bar(AdjMarkers<T> am, const T *rb0, const T *rb1, const T *rb2, T dt_rho) {
  AdjRow<T, DIM> L(am, 1);
  T s = T(0), sd[3] = {T(0), T(0), T(0)};
  if (L.valid) {
    const T *rc = L.c == 0 ? rb0 : (L.c == 1 ? rb1 : rb2);
    T r4[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) r4[j] = rc[L.node[j]];
    T sx = T(0), sdx = T(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      sx += r4[j] * L.wx[j];
      sdx += r4[j] * L.dwx[j];
    }
    s = sx * L.wy * L.wz;
    sd[0] = sdx * L.wy * L.wz;
    sd[1] = sx * L.dwy * L.wz;
    if (DIM == 3) sd[2] = sx * L.wy * L.dwz;
  }
  s = group_sum<AdjRow<T, DIM>::ROWS>(s);
#pragma unroll
  for (int a = 0; a < DIM; ++a) sd[a] = group_sum<AdjRow<T, DIM>::ROWS>(sd[a]);
  if (L.valid && L.jy == 0 && L.kz == 0) {
    const T scale = dt_rho * (T)am.inv_vol;
    am.Gb[L.c][L.k] = s * scale;
    const T g = am.G[L.c][L.k] * scale;
#pragma unroll
    for (int a = 0; a < DIM; ++a) atomicAdd(am.Xhb[a] + L.k, (double)(g * sd[a]));
  }
}

// 2a adjoint (zero rest length): Xhb_a += sum_b kappa (Gb_b - Gb_a);
// d(loss)/d kappa_e += (Xh_b - Xh_a).(Gb_a - Gb_b), counted once per
// connection (from its CSR entry with a < b).  8 lanes per marker share its
// CSR row (lane j takes entries j, j + 8, ...) and reduce with shuffles.
template <typename T, int DIM>
__global__ void k_adj_force_bar(AdjMarkers<T> am) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long a = t >> 3;
  const int lane8 = (int)(t & 7);
  const bool valid = a < am.nm;
  double acc[DIM];
#pragma unroll
  for (int q = 0; q < DIM; ++q) acc[q] = 0.0;
  if (valid) {
    double xa[DIM];
    T ga[DIM];
#pragma unroll
    for (int q = 0; q < DIM; ++q) {
      xa[q] = am.Xh[q][a];
      ga[q] = am.Gb[q][a];
    }
    for (long long e = am.row[a] + lane8; e < am.row[a + 1]; e += 8) {
      const int b = am.col[e];
      const double kap = am.kap[e];
      double dot = 0.0;
#pragma unroll
      for (int q = 0; q < DIM; ++q) {
        const double gb = (double)am.Gb[q][b];
        acc[q] += kap * (gb - (double)ga[q]);
        double d = am.Xh[q][b] - xa[q];
        d -= am.H * rint(d / am.H);
        dot += d * ((double)ga[q] - gb);
      }
      if (b > a) am.dk[am.cedge[e]] += dot;
    }
  }
#pragma unroll
  for (int q = 0; q < DIM; ++q)
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
  if (valid && lane8 == 0) {
#pragma unroll
    for (int q = 0; q < DIM; ++q) am.Xhb[q][a] += acc[q];
  }
}

// 1b-1c adjoint: Xb <- Xb + Xhb; vbar = dt Xb' + dt/2 Xhb;
// Ub = c1 vbar + Uoldb'; Uoldb = c2 vbar
template <typename T, int DIM>
__global__ void k_adj_update_bar(AdjMarkers<T> am) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= am.nm * DIM) return;
  const long long k = t / DIM;
  const int c = (int)(t % DIM);
  const double xb = am.Xb[c][k], xhb = am.Xhb[c][k];
  const double vb = am.dt * xb + 0.5 * am.dt * xhb;
  am.Xb[c][k] = xb + xhb;
  const double c1 = am.first ? 1.0 : 1.5, c2 = am.first ? 0.0 : -0.5;
  am.Ub[c][k] = (T)(c1 * vb + (double)am.Uoldb[c][k]);
  am.Uoldb[c][k] = (T)(c2 * vb);
}

// 1a adjoint: ub_c += Ub_c W (spreading without 1/h^d); Xb_a += Ub_c sum u_c dW/dX_a
template <typename T, int DIM>
__global__ void k_adj_interp_bar(AdjMarkers<T> am, const T *u0, const T *u1, const T *u2, T *ub0, T *ub1, T *ub2) {
  AdjRow<T, DIM> L(am, 0);
  T sd[3] = {T(0), T(0), T(0)};
  T Ub = T(0);
  if (L.valid) {
    const T *uc = L.c == 0 ? u0 : (L.c == 1 ? u1 : u2);
    T *ubc = L.c == 0 ? ub0 : (L.c == 1 ? ub1 : ub2);
    Ub = am.Ub[L.c][L.k];
    const T wr = L.wy * L.wz;
    T sx = T(0), sdx = T(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      atomicAdd(ubc + L.node[j], Ub * (L.wx[j] * wr));
      const T un = uc[L.node[j]];
      sx += un * L.wx[j];
      sdx += un * L.dwx[j];
    }
    sd[0] = sdx * wr;
    sd[1] = sx * L.dwy * L.wz;
    if (DIM == 3) sd[2] = sx * L.wy * L.dwz;
  }
#pragma unroll
  for (int a = 0; a < DIM; ++a) sd[a] = group_sum<AdjRow<T, DIM>::ROWS>(sd[a]);
  if (L.valid && L.jy == 0 && L.kz == 0)
#pragma unroll
    for (int a = 0; a < DIM; ++a) atomicAdd(am.Xb[a] + L.k, (double)(Ub * sd[a]));
}

// --------------------------------------------------------------------------

static inline unsigned nb(long long work) {
  long long b = (work + 255) / 256;
  const long long sms = device_sms(), cap = (sms > 0 ? sms : 152) * 16;
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename T>
cudaError_t adjoint_fields_a(const AdjFields<T> &f, cudaStream_t s) {
  k_adj_q<T><<<nb(f.cells), 256, 0, s>>>(f.psib, f.pb, f.q, f.cells);
  return cudaGetLastError();
}

template <typename T>
cudaError_t adjoint_fields_b(const AdjFields<T> &f, cudaStream_t s) {
  k_adj_div<T><<<nb(f.cells), 256, 0, s>>>(f.q, f.divb, f.pb, f.chi_mu_half, f.rho_dt, f.p_keep, f.cells);
  if (f.dim == 2)
    k_adj_grad<T, 2><<<dim3((f.n[0] + 127) / 128, f.n[1], 1), 128, 0, s>>>(
        f.ub[0], f.ub[1], f.ub[1], f.rb[0], f.rb[1], f.rb[1], f.q, f.n[0], f.n[1], 1, f.ih[0], f.ih[1], T(0));
  else
    k_adj_grad<T, 3><<<dim3((f.n[0] + 127) / 128, f.n[1], f.n[2]), 128, 0, s>>>(
        f.ub[0], f.ub[1], f.ub[2], f.rb[0], f.rb[1], f.rb[2], f.q, f.n[0], f.n[1], f.n[2], f.ih[0], f.ih[1],
        f.ih[2]);
  return cudaGetLastError();
}

template <typename T>
cudaError_t adjoint_fields_c(const AdjFields<T> &f, const T *const u[3], int first, cudaStream_t s) {
  if (f.dim == 2) {
    k_adj_rhs<T, 2><<<dim3((f.n[0] + 127) / 128, f.n[1], 1), 128, 0, s>>>(
        f.ub[0], f.ub[1], f.ub[1], f.rb[0], f.rb[1], f.rb[1], f.nbar[0],
                                                f.nbar[1], f.nbar[1], f.vv[0], f.vv[1], f.vv[1], f.pb, f.psib, f.n[0],
                                                f.n[1], 1, f.ih[0], f.ih[1], T(0), f.dt_mu_rho, f.dt_rho, f.dt, f.psi_w,
                                                first);
    k_adj_adv<T, 2><<<dim3((f.n[0] + 127) / 128, f.n[1], 1), 128, 0, s>>>(
        f.ub[0], f.ub[1], f.ub[1], u[0], u[1], u[1], f.vv[0], f.vv[1], f.vv[1], f.n[0], f.n[1], 1, f.ih[0], f.ih[1],
        T(0));
  } else {
    k_adj_rhs<T, 3><<<dim3((f.n[0] + 127) / 128, f.n[1], f.n[2]), 128, 0, s>>>(
        f.ub[0], f.ub[1], f.ub[2], f.rb[0], f.rb[1], f.rb[2], f.nbar[0],
                                                f.nbar[1], f.nbar[2], f.vv[0], f.vv[1], f.vv[2], f.pb, f.psib, f.n[0],
                                                f.n[1], f.n[2], f.ih[0], f.ih[1], f.ih[2], f.dt_mu_rho, f.dt_rho,
                                                f.dt, f.psi_w, first);
    k_adj_adv<T, 3><<<dim3((f.n[0] + 127) / 128, f.n[1], f.n[2]), 128, 0, s>>>(
        f.ub[0], f.ub[1], f.ub[2], u[0], u[1], u[2], f.vv[0], f.vv[1], f.vv[2], f.n[0], f.n[1], f.n[2], f.ih[0],
        f.ih[1], f.ih[2]);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t adjoint_markers_pre(const AdjMarkers<T> &am, const T *const u[3], cudaStream_t s) {
  if (am.nm == 0) return cudaSuccess;
  const unsigned g = (unsigned)((am.nm * am.dim + 255) / 256);
  const unsigned gr = (unsigned)((am.nm * am.dim * (am.dim == 3 ? 16 : 4) + 255) / 256);
  if (am.dim == 2) {
    k_adj_stencil<T, 2><<<g, 256, 0, s>>>(am, 0);
    k_adj_interp_fwd<T, 2><<<gr, 256, 0, s>>>(am, u[0], u[1], u[1]);
    k_adj_half<T, 2><<<g, 256, 0, s>>>(am);
  } else {
    k_adj_stencil<T, 3><<<g, 256, 0, s>>>(am, 0);
    k_adj_interp_fwd<T, 3><<<gr, 256, 0, s>>>(am, u[0], u[1], u[2]);
    k_adj_half<T, 3><<<g, 256, 0, s>>>(am);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t adjoint_markers_post(const AdjMarkers<T> &am, const T *const rb[3], T dt_rho, const T *const u[3],
                                 T *const ub[3], cudaStream_t s) {
  if (am.nm == 0) return cudaSuccess;
  const unsigned g = (unsigned)((am.nm * am.dim + 255) / 256), g8 = (unsigned)((am.nm * 8 + 255) / 256);
  const unsigned gr = (unsigned)((am.nm * am.dim * (am.dim == 3 ? 16 : 4) + 255) / 256);
  if (am.dim == 2) {
    k_adj_stencil<T, 2><<<g, 256, 0, s>>>(am, 1);
    k_adj_spread_bar<T, 2><<<gr, 256, 0, s>>>(am, rb[0], rb[1], rb[1], dt_rho);
    k_adj_force_bar<T, 2><<<g8, 256, 0, s>>>(am);
    k_adj_update_bar<T, 2><<<g, 256, 0, s>>>(am);
    k_adj_interp_bar<T, 2><<<gr, 256, 0, s>>>(am, u[0], u[1], u[1], ub[0], ub[1], ub[1]);
  } else {
    k_adj_stencil<T, 3><<<g, 256, 0, s>>>(am, 1);
    k_adj_spread_bar<T, 3><<<gr, 256, 0, s>>>(am, rb[0], rb[1], rb[2], dt_rho);
    k_adj_force_bar<T, 3><<<g8, 256, 0, s>>>(am);
    k_adj_update_bar<T, 3><<<g, 256, 0, s>>>(am);
    k_adj_interp_bar<T, 3><<<gr, 256, 0, s>>>(am, u[0], u[1], u[2], ub[0], ub[1], ub[2]);
  }
  return cudaGetLastError();
}

#define IBG_ADJ_INST(T)                                                                                       \
  template cudaError_t adjoint_fields_a<T>(const AdjFields<T> &, cudaStream_t);                               \
  template cudaError_t adjoint_fields_b<T>(const AdjFields<T> &, cudaStream_t);                               \
  template cudaError_t adjoint_fields_c<T>(const AdjFields<T> &, const T *const[3], int, cudaStream_t);       \
  template cudaError_t adjoint_markers_pre<T>(const AdjMarkers<T> &, const T *const[3], cudaStream_t);        \
  template cudaError_t adjoint_markers_post<T>(const AdjMarkers<T> &, const T *const[3], T, const T *const[3], \
                                               T *const[3], cudaStream_t);
IBG_ADJ_INST(float)
IBG_ADJ_INST(double)

}  // namespace ibg
