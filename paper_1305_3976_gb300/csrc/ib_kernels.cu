// Marker kernels (Steps 1a-2b), the explicit momentum right-hand side
// (Steps 3a-3b), the divergence and the FP64 diagnostics, for sm_103a.
#include <math.h>

#include "ib_internal.cuh"

namespace ibg {

// ---------------------------------------------------------------------------
// 1D kernel weights.  For a node offset o (0 on the component's own axis,
// 1/2 elsewhere) put x = X/h - o, i0 = floor(x), f = x - i0; the four nodes
// i0-1 .. i0+2 sit at r = -1-f, -f, 1-f, 2-f.  Both branches of the 4-point
// kernel of eq. (discretedelta) share q = sqrt(1 + 4f - 4f^2) on these four
// nodes, which gives the weights (3-2f-q)/8, (3-2f+q)/8, (1+2f+q)/8,
// (1+2f-q)/8 (they sum to 1).  The cosine kernel is (1 + cos(pi r / 2)) / 4.
// Positions are FP64; the weights are computed in the field precision T.

__device__ __forceinline__ float cospi_t(float x) { return cospif(x); }
__device__ __forceinline__ double cospi_t(double x) { return cospi(x); }

template <typename T>
__device__ __forceinline__ long long delta_weights(double X, double inv_h, double off, int kernel, T (&w)[4]) {
  const double x = X * inv_h - off;
  const double fl = floor(x);
  const T f = (T)(x - fl);
  if (kernel == 0) {
    const T q = sqrt(T(1) + T(4) * f * (T(1) - f));
    const T a = T(3) - T(2) * f, b = T(1) + T(2) * f;
    w[0] = (a - q) * T(0.125);
    w[1] = (a + q) * T(0.125);
    w[2] = (b + q) * T(0.125);
    w[3] = (b - q) * T(0.125);
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) w[j] = T(0.25) * (T(1) + cospi_t((T(j - 1) - f) * T(0.5)));
  }
  return (long long)fl - 1;
}

__device__ __forceinline__ int wrap_idx(long long i, int n) {
  long long r = i % n;
  return (int)(r < 0 ? r + n : r);
}

// Step 1a + Steps 1b-1c: one thread per (marker, component c).
//   U_c = sum over the 4^d nodes of u_c(node) prod_a phi_a
//   X^{n+1/2}_c = 1/2 ((X_c + dt V_c) + X_c),  V = 3/2 U^n - 1/2 U^{n-1}
//   (V = U^0 at n = 0).  X^{n+1} is written by the force kernel.
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_interp(const MarkerArgs m, const T *const u0, const T *const u1,
                                                const T *const u2) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.nm * DIM) return;
  const long long k = t / DIM;
  const int c = (int)(t % DIM);
  const T *uc = c == 0 ? u0 : (c == 1 ? u1 : u2);
  const int nx = m.n[0], ny = m.n[1];
  T w[3][4];
  int idx[3][4];
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const long long b = delta_weights<T>(m.X[a][k], m.inv_h[a], a == c ? 0.0 : 0.5, m.kernel, w[a]);
#pragma unroll
    for (int j = 0; j < 4; ++j) idx[a][j] = wrap_idx(b + j, m.n[a]);
  }
  T s = T(0);
  if (DIM == 2) {
#pragma unroll
    for (int jy = 0; jy < 4; ++jy) {
      const T *row = uc + (long long)idx[1][jy] * nx;
#pragma unroll
      for (int ix = 0; ix < 4; ++ix) s += __ldg(row + idx[0][ix]) * (w[0][ix] * w[1][jy]);
    }
  } else {
#pragma unroll
    for (int kz = 0; kz < 4; ++kz)
#pragma unroll
      for (int jy = 0; jy < 4; ++jy) {
        const T *row = uc + ((long long)idx[2][kz] * ny + idx[1][jy]) * nx;
        const T wyz = w[1][jy] * w[2][kz];
#pragma unroll
        for (int ix = 0; ix < 4; ++ix) s += __ldg(row + idx[0][ix]) * (w[0][ix] * wyz);
      }
  }
  const double U = (double)s;
  const double vel = m.first ? U : 1.5 * U - 0.5 * m.Uold[c][k];
  const double Xc = m.X[c][k];
  m.Xh[c][k] = 0.5 * ((Xc + m.dt * vel) + Xc);
  m.U[c][k] = U;
}

// Step 2a over the force connections at X^{n+1/2} (CSR by marker), then the
// marker update X^{n+1} = X^n + dt V of Step 1b.  One thread per (marker, c).
template <int DIM>
__global__ void __launch_bounds__(256) k_force(const MarkerArgs m) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.nm * DIM) return;
  const long long a = t / DIM;
  const int c = (int)(t % DIM);
  double xa[DIM];
#pragma unroll
  for (int q = 0; q < DIM; ++q) xa[q] = m.Xh[q][a];
  double g = 0.0;
  for (long long e = m.row[a]; e < m.row[a + 1]; ++e) {
    const int b = m.col[e];
    double d[DIM], len2 = 0.0;
#pragma unroll
    for (int q = 0; q < DIM; ++q) {
      d[q] = m.Xh[q][b] - xa[q];
      d[q] -= m.H * round(d[q] / m.H);  // nearest periodic image
      len2 += d[q] * d[q];
    }
    double scale = m.kap[e];
    const double L = m.rest[e];
    if (L != 0.0) scale *= 1.0 - L / sqrt(len2);
    g += scale * d[c];
  }
  m.G[c][a] = g;
  const double U = m.U[c][a];
  const double vel = m.first ? U : 1.5 * U - 0.5 * m.Uold[c][a];
  m.X[c][a] = m.X[c][a] + m.dt * vel;
  m.Uold[c][a] = U;
}

// Step 2b: f_c(node) += G_c prod_a phi_a / h^d with atomics.  One thread per
// (marker, c); the 4 nodes along x of a row are contiguous.
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_spread(const MarkerArgs m, T *const f0, T *const f1, T *const f2) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.nm * DIM) return;
  const long long k = t / DIM;
  const int c = (int)(t % DIM);
  T *fc = c == 0 ? f0 : (c == 1 ? f1 : f2);
  const int nx = m.n[0], ny = m.n[1];
  T w[3][4];
  int idx[3][4];
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const long long b = delta_weights<T>(m.Xh[a][k], m.inv_h[a], a == c ? 0.0 : 0.5, m.kernel, w[a]);
#pragma unroll
    for (int j = 0; j < 4; ++j) idx[a][j] = wrap_idx(b + j, m.n[a]);
  }
  const T val = (T)(m.G[c][k] * m.inv_vol);
  if (DIM == 2) {
#pragma unroll
    for (int jy = 0; jy < 4; ++jy) {
      T *row = fc + (long long)idx[1][jy] * nx;
      const T vy = val * w[1][jy];
#pragma unroll
      for (int ix = 0; ix < 4; ++ix) atomicAdd(row + idx[0][ix], vy * w[0][ix]);
    }
  } else {
#pragma unroll
    for (int kz = 0; kz < 4; ++kz)
#pragma unroll
      for (int jy = 0; jy < 4; ++jy) {
        T *row = fc + ((long long)idx[2][kz] * ny + idx[1][jy]) * nx;
        const T vyz = val * (w[1][jy] * w[2][kz]);
#pragma unroll
        for (int ix = 0; ix < 4; ++ix) atomicAdd(row + idx[0][ix], vyz * w[0][ix]);
      }
  }
}

// ---------------------------------------------------------------------------
// Steps 3a-3b in increment form: R_c = u*_c - u^n_c
//   = dt [ (mu L u_c - G_c p* + f_c) / rho - (3/2 N_c(u^n) - 1/2 N_c(u^{n-1})) ]
// with p* = p^{n-1/2} + psi^{n-1/2} (0 at n = 0) and N^{1/2} = N(u^0).
// N is the skew-symmetric form (1/2 u.grad u + 1/2 div(uu)) on the staggered
// grid: along each axis a the divergence and advective halves with one shared
// transport velocity A+- (the a-velocity averaged to the two flux points half
// a cell above and below the c-face) add up to 1/2 (A+ u_c(+a) - A- u_c(-a))/h_a.
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_rhs(const RhsArgs<T> a) {
  const int nx = a.n[0], ny = a.n[1], nz = DIM == 3 ? a.n[2] : 1;
  const long long cells = (long long)nx * ny * nz;
  for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < cells;
       o += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(o % nx);
    const long long tq = o / nx;
    const int j = (int)(tq % ny);
    const int k = (int)(tq / ny);
    long long dp[3], dm[3];
    dp[0] = i + 1 == nx ? 1 - nx : 1;
    dm[0] = i == 0 ? nx - 1 : -1;
    dp[1] = j + 1 == ny ? (long long)nx * (1 - ny) : nx;
    dm[1] = j == 0 ? (long long)nx * (ny - 1) : -(long long)nx;
    if (DIM == 3) {
      const long long pl = (long long)nx * ny;
      dp[2] = k + 1 == nz ? pl * (1 - nz) : pl;
      dm[2] = k == 0 ? pl * (nz - 1) : -pl;
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const T *uc = a.u[c];
      const T u0 = uc[o];
      T lap = T(0), adv = T(0);
#pragma unroll
      for (int ax = 0; ax < DIM; ++ax) {
        const T up = uc[o + dp[ax]], um = uc[o + dm[ax]];
        lap += (up - T(2) * u0 + um) * a.inv_h2[ax];
        T Ap, Am;
        if (ax == c) {
          Ap = T(0.5) * (u0 + up);
          Am = T(0.5) * (um + u0);
        } else {
          const T *ua = a.u[ax];
          Ap = T(0.5) * (ua[o + dp[ax]] + ua[o + dp[ax] + dm[c]]);
          Am = T(0.5) * (ua[o] + ua[o + dm[c]]);
        }
        adv += T(0.5) * (Ap * up - Am * um) * a.inv_h[ax];
      }
      T gp = T(0);
      if (!a.first) gp = ((a.p[o] + a.psi[o]) - (a.p[o + dm[c]] + a.psi[o + dm[c]])) * a.inv_h[c];
      const T Nh = a.first ? adv : T(1.5) * adv - T(0.5) * a.Nold[c][o];
      const T f = a.scr[c][o];
      a.scr[c][o] = a.dt * ((a.mu * lap - gp + f) * a.inv_rho - Nh);
      a.Nold[c][o] = adv;
    }
  }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_divergence(const T *u0, const T *u1, const T *u2, T *div, int nx, int ny,
                                                    int nz, T ihx, T ihy, T ihz) {
  const long long cells = (long long)nx * ny * nz;
  for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < cells;
       o += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(o % nx);
    const long long tq = o / nx;
    const int j = (int)(tq % ny);
    const int k = (int)(tq / ny);
    T d = (u0[o + (i + 1 == nx ? 1 - nx : 1)] - u0[o]) * ihx;
    d += (u1[o + (j + 1 == ny ? (long long)nx * (1 - ny) : nx)] - u1[o]) * ihy;
    if (DIM == 3) d += (u2[o + (k + 1 == nz ? (long long)nx * ny * (1 - nz) : (long long)nx * ny)] - u2[o]) * ihz;
    div[o] = d;
  }
}

// ---------------------------------------------------------------------------
// FP64 diagnostics: block reductions, one double atomic per block and value.
// acc[0] sum div^2, acc[1] max |div|, acc[2] sum |u|^2, acc[3] volume,
// acc[4] elastic energy, acc[5] count of non-finite values.

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
  // for v >= 0 the IEEE bit pattern orders like a signed integer
  atomicMax(reinterpret_cast<long long *>(addr), __double_as_longlong(v));
}

template <int NV>
__device__ void block_reduce_add(double (&v)[NV], double *acc, const int *slot, int maxslot) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double x = (slot[q] == maxslot) ? warp_max(v[q]) : warp_sum(v[q]);
    if (lane == 0) sh[q][w] = x;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double x = lane < nw ? sh[q][lane] : 0.0;
      x = (slot[q] == maxslot) ? warp_max(x) : warp_sum(x);
      if (lane == 0) {
        if (slot[q] == maxslot) atomic_max_nonneg(acc + slot[q], x);
        else atomicAdd(acc + slot[q], x);
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_field_diag(int dim, const T *u0, const T *u1, const T *u2, const T *p,
                                                    const T *div, long long cells, double *acc) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < cells;
       o += (long long)gridDim.x * blockDim.x) {
    const double d = (double)div[o];
    const double a = (double)u0[o], b = (double)u1[o], c = dim == 3 ? (double)u2[o] : 0.0;
    const double pp = (double)p[o];
    v[0] += d * d;
    v[1] = fmax(v[1], fabs(d));
    v[2] += a * a + b * b + c * c;
    if (!isfinite(d) || !isfinite(a) || !isfinite(b) || !isfinite(c) || !isfinite(pp)) v[3] += 1.0;
  }
  const int slot[4] = {0, 1, 2, 5};
  block_reduce_add<4>(v, acc, slot, 1);
}

__global__ void __launch_bounds__(256) k_marker_diag(int dim, const double *X0, const double *X1, const double *X2,
                                                     long long nm, const int32_t *edges, const double *kappa,
                                                     const double *rest, long long ne, const int32_t *tris,
                                                     long long nt, double H, double *acc) {
  double v[3] = {0.0, 0.0, 0.0};
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long e = t0; e < ne; e += stride) {
    const int a = edges[2 * e], b = edges[2 * e + 1];
    const double dx = X0[b] - X0[a], dy = X1[b] - X1[a], dz = dim == 3 ? X2[b] - X2[a] : 0.0;
    double ddx = dx - H * round(dx / H), ddy = dy - H * round(dy / H), ddz = dz - H * round(dz / H);
    const double ext = sqrt(ddx * ddx + ddy * ddy + ddz * ddz) - rest[e];
    v[1] += 0.5 * kappa[e] * ext * ext;
    if (dim == 2) v[0] += 0.5 * (X0[a] * X1[b] - X0[b] * X1[a]);  // directed edge loop area
  }
  if (dim == 3) {
    for (long long q = t0; q < nt; q += stride) {
      const int a = tris[3 * q], b = tris[3 * q + 1], c = tris[3 * q + 2];
      const double ax = X0[a], ay = X1[a], az = X2[a], bx = X0[b], by = X1[b], bz = X2[b];
      const double cx = X0[c], cy = X1[c], cz = X2[c];
      v[0] += (ax * (by * cz - bz * cy) - ay * (bx * cz - bz * cx) + az * (bx * cy - by * cx)) / 6.0;
    }
  }
  for (long long q = t0; q < nm; q += stride) {
    const double x = X0[q] + X1[q] + (dim == 3 ? X2[q] : 0.0);
    if (!isfinite(x)) v[2] += 1.0;
  }
  const int slot[3] = {3, 4, 5};
  block_reduce_add<3>(v, acc, slot, -1);
}

// marker positions between the caller's [n][dim] layout and the SoA arrays
__global__ void __launch_bounds__(256) k_markers_layout(double *aos, double *X0, double *X1, double *X2,
                                                        long long nm, int dim, int to_soa) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nm * dim) return;
  const long long k = t / dim;
  const int c = (int)(t % dim);
  double *X = c == 0 ? X0 : (c == 1 ? X1 : X2);
  if (to_soa) X[k] = aos[t];
  else aos[t] = X[k];
}

// ---------------------------------------------------------------------------
// launchers

static inline unsigned blocks_for(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : b);
}
static inline unsigned grid_stride_blocks(long long work) {
  // enough CTAs for every SM of a GB300 several times over, then grid-stride
  long long b = (work + 255) / 256;
  const long long cap = 152 * 16;
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename T>
cudaError_t launch_interp(const MarkerArgs &m, const T *const u[3], cudaStream_t s) {
  if (m.nm == 0) return cudaSuccess;
  const unsigned g = blocks_for(m.nm * m.dim, 256);
  if (m.dim == 2) k_interp<T, 2><<<g, 256, 0, s>>>(m, u[0], u[1], u[1]);
  else k_interp<T, 3><<<g, 256, 0, s>>>(m, u[0], u[1], u[2]);
  return cudaGetLastError();
}

cudaError_t launch_force(const MarkerArgs &m, cudaStream_t s) {
  if (m.nm == 0) return cudaSuccess;
  const unsigned g = blocks_for(m.nm * m.dim, 256);
  if (m.dim == 2) k_force<2><<<g, 256, 0, s>>>(m);
  else k_force<3><<<g, 256, 0, s>>>(m);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spread(const MarkerArgs &m, T *const f[3], cudaStream_t s) {
  if (m.nm == 0) return cudaSuccess;
  const unsigned g = blocks_for(m.nm * m.dim, 256);
  if (m.dim == 2) k_spread<T, 2><<<g, 256, 0, s>>>(m, f[0], f[1], f[1]);
  else k_spread<T, 3><<<g, 256, 0, s>>>(m, f[0], f[1], f[2]);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rhs(int dim, const RhsArgs<T> &a, cudaStream_t s) {
  const long long cells = (long long)a.n[0] * a.n[1] * (dim == 3 ? a.n[2] : 1);
  const unsigned g = grid_stride_blocks(cells);
  if (dim == 2) k_rhs<T, 2><<<g, 256, 0, s>>>(a);
  else k_rhs<T, 3><<<g, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_divergence(int dim, const T *const u[3], T *div, const int n[3], const T inv_h[3],
                              cudaStream_t s) {
  const int nz = dim == 3 ? n[2] : 1;
  const long long cells = (long long)n[0] * n[1] * nz;
  const unsigned g = grid_stride_blocks(cells);
  if (dim == 2) k_divergence<T, 2><<<g, 256, 0, s>>>(u[0], u[1], u[1], div, n[0], n[1], 1, inv_h[0], inv_h[1], T(0));
  else k_divergence<T, 3><<<g, 256, 0, s>>>(u[0], u[1], u[2], div, n[0], n[1], nz, inv_h[0], inv_h[1], inv_h[2]);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_field_diag(int dim, const T *const u[3], const T *p, const T *div, const int n[3], double *acc,
                              cudaStream_t s) {
  const long long cells = (long long)n[0] * n[1] * (dim == 3 ? n[2] : 1);
  k_field_diag<T><<<grid_stride_blocks(cells), 256, 0, s>>>(dim, u[0], u[1], dim == 3 ? u[2] : u[1], p, div,
                                                            cells, acc);
  return cudaGetLastError();
}

cudaError_t launch_marker_diag(int dim, const double *const X[3], int64_t nm, const int32_t *edges,
                               const double *kappa, const double *rest, int64_t ne, const int32_t *tris,
                               int64_t nt, double H, double *acc, cudaStream_t s) {
  long long work = nm > ne ? nm : ne;
  if (nt > work) work = nt;
  if (work == 0) return cudaSuccess;
  k_marker_diag<<<grid_stride_blocks(work), 256, 0, s>>>(dim, X[0], X[1], dim == 3 ? X[2] : X[1], nm, edges, kappa,
                                                         rest, ne, tris, nt, H, acc);
  return cudaGetLastError();
}

cudaError_t launch_markers_layout(double *aos, double *const X[3], int64_t nm, int dim, int to_soa,
                                  cudaStream_t s) {
  if (nm == 0) return cudaSuccess;
  k_markers_layout<<<blocks_for(nm * dim, 256), 256, 0, s>>>(aos, X[0], X[1], X[2], nm, dim, to_soa);
  return cudaGetLastError();
}

template cudaError_t launch_interp<float>(const MarkerArgs &, const float *const[3], cudaStream_t);
template cudaError_t launch_interp<double>(const MarkerArgs &, const double *const[3], cudaStream_t);
template cudaError_t launch_spread<float>(const MarkerArgs &, float *const[3], cudaStream_t);
template cudaError_t launch_spread<double>(const MarkerArgs &, double *const[3], cudaStream_t);
template cudaError_t launch_rhs<float>(int, const RhsArgs<float> &, cudaStream_t);
template cudaError_t launch_rhs<double>(int, const RhsArgs<double> &, cudaStream_t);
template cudaError_t launch_divergence<float>(int, const float *const[3], float *, const int[3], const float[3],
                                              cudaStream_t);
template cudaError_t launch_divergence<double>(int, const double *const[3], double *, const int[3], const double[3],
                                               cudaStream_t);
template cudaError_t launch_field_diag<float>(int, const float *const[3], const float *, const float *, const int[3],
                                              double *, cudaStream_t);
template cudaError_t launch_field_diag<double>(int, const double *const[3], const double *, const double *,
                                               const int[3], double *, cudaStream_t);

}  // namespace ibg
