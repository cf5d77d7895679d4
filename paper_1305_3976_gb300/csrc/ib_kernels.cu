// The explicit momentum right-hand side (Steps 3a-3b), the divergence and
// the FP64 diagnostics, for sm_103a.
#include <math.h>

#include <vector>

#include "ib_internal.cuh"

namespace ibg {

// ---------------------------------------------------------------------------
// Steps 3a-3b in increment form: R_c = u*_c - u^n_c
//   = dt [ (mu L u_c - G_c p* + f_c) / rho - (3/2 N_c(u^n) - 1/2 N_c(u^{n-1})) ]
// with p* = p^{n-1/2} + psi^{n-1/2} (0 at n = 0) and N^{1/2} = N(u^0).
// The kernels below store R without the force term; the spreading kernel,
// which runs after them, adds dt/rho f_c into R.
// N is the skew-symmetric form (1/2 u.grad u + 1/2 div(uu)) on the staggered
// grid: along each axis a the divergence and advective halves with one shared
// transport velocity A+- (the a-velocity averaged to the two flux points half
// a cell above and below the c-face) add up to 1/2 (A+ u_c(+a) - A- u_c(-a))/h_a.
template <typename T, int DIM>
__device__ __forceinline__ void rhs_body(const RhsArgs<T> &a, const Blk &B) {
  const int nx = a.n[0], ny = a.n[1], nz = DIM == 3 ? a.n[2] : 1;
  const long long cells = (long long)nx * ny * nz;
  // cell counts stay below 2^31 (n <= 512 per axis): 32-bit index arithmetic
  for (unsigned o = B.x * blockDim.x + threadIdx.x; o < (unsigned)cells; o += B.gx * blockDim.x) {
    const int i = (int)(o % (unsigned)nx);
    const unsigned tq = o / (unsigned)nx;
    const int j = (int)(tq % (unsigned)ny);
    const int k = (int)(tq / (unsigned)ny);
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
    // every load first (the stores below may alias nothing the compiler can see)
    T uc[DIM], up[DIM][DIM], um[DIM][DIM], ux[DIM][DIM];  // ux[c][a] = u_a at face + e_a - e_c
    T nold[DIM], pm[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const T *u = a.u[c];
      uc[c] = u[o];
#pragma unroll
      for (int ax = 0; ax < DIM; ++ax) {
        up[c][ax] = u[o + dp[ax]];
        um[c][ax] = u[o + dm[ax]];
      }
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c)
#pragma unroll
      for (int ax = 0; ax < DIM; ++ax) ux[c][ax] = ax == c ? T(0) : a.u[ax][o + dp[ax] + dm[c]];
    const T p0 = a.first ? T(0) : a.p[o] + (a.psi ? a.psi[o] : T(0));
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      nold[c] = a.first ? T(0) : a.Nold[c][o];
      pm[c] = a.first ? T(0) : a.p[o + dm[c]] + (a.psi ? a.psi[o + dm[c]] : T(0));
    }
    // per axis: 1/2 (A+ u(+a) - A- u(-a)) / h_a with A+- the averages of two
    // velocities is (1 / (4 h_a)) ((a0 + a1) u(+a) - (b0 + b1) u(-a)); the
    // Laplacian sums (u(+a) + u(-a)) / h_a^2 and subtracts 2 u sum_a 1/h_a^2
    T q4[DIM], s2 = T(0);
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
      q4[ax] = T(0.25) * a.inv_h[ax];
      s2 += a.inv_h2[ax];
    }
    T R[DIM], Nn[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      T lap = T(-2) * s2 * uc[c], adv = T(0);
#pragma unroll
      for (int ax = 0; ax < DIM; ++ax) {
        lap = fma(up[c][ax] + um[c][ax], a.inv_h2[ax], lap);
        T sp, sm;
        if (ax == c) {
          sp = uc[c] + up[c][ax];
          sm = um[c][ax] + uc[c];
        } else {
          sp = up[ax][ax] + ux[c][ax];   // u_a at +e_a and at +e_a - e_c
          sm = uc[ax] + um[ax][c];       // u_a at the face and at -e_c
        }
        adv = fma(q4[ax], sp * up[c][ax] - sm * um[c][ax], adv);
      }
      // dt mu/rho L u - dt/rho G p* - dt (3/2 N^n - 1/2 N^{n-1}) (n == 0: - dt N^0)
      T acc = a.cmu * lap;
      acc = fma(a.ncg[c], p0 - pm[c], acc);
      acc = fma(a.ncA, adv, acc);
      R[c] = fma(a.cN, nold[c], acc);
      Nn[c] = adv;
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      a.scr[c][o] = R[c];
      a.Nold[c][o] = Nn[c];
    }
  }
}
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_rhs(const RhsArgs<T> a) {
  pdl_wait();
  pdl_release();
  rhs_body<T, DIM>(a, hw_blk());
}
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_rhs_b(const __grid_constant__ Batch<RhsArgs<T>> Bt) {
  pdl_wait();
  pdl_release();
  Blk b;
  const int i = batch_member(Bt, b);
  rhs_body<T, DIM>(Bt.a[i], b);
}

// 4 values of a row at x0 + shift .. x0 + 3 + shift (shift in {-1, 0, 1}),
// periodic in x: one 128-bit load plus at most one single load
template <typename T>
__device__ __forceinline__ void get4(const T *f, int ro, int x0, int nx, int shift, T (&v)[4]) {
  T c[4];
  ld4(f + ro + x0, c);
  if (shift == 0) {
    v[0] = c[0]; v[1] = c[1]; v[2] = c[2]; v[3] = c[3];
  } else if (shift < 0) {
    v[0] = f[ro + (x0 == 0 ? nx - 1 : x0 - 1)];
    v[1] = c[0]; v[2] = c[1]; v[3] = c[2];
  } else {
    v[0] = c[1]; v[1] = c[2]; v[2] = c[3];
    v[3] = f[ro + (x0 + 4 == nx ? 0 : x0 + 4)];
  }
}

// component C of the right-hand side at 4 consecutive x cells
template <typename T, int DIM, int C>
__device__ __forceinline__ void rhs4_component(const RhsArgs<T> &a, int x0, int y, int z) {
  const int nx = a.n[0], ny = a.n[1], nz = DIM == 3 ? a.n[2] : 1;
  const int yp = y + 1 == ny ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
  const int zp = z + 1 == nz ? 0 : z + 1, zm = z == 0 ? nz - 1 : z - 1;
  auto R = [&](int yy, int zz) { return (zz * ny + yy) * nx; };
  const int ro = R(y, z);
  // u_C: centre and the 6 neighbours (dir 1/2 = +x/-x, 3/4 = +y/-y, 5/6 = +z/-z)
  T S[7][4];
  get4(a.u[C], ro, x0, nx, 0, S[0]);
  get4(a.u[C], ro, x0, nx, 1, S[1]);
  get4(a.u[C], ro, x0, nx, -1, S[2]);
  get4(a.u[C], R(yp, z), x0, nx, 0, S[3]);
  get4(a.u[C], R(ym, z), x0, nx, 0, S[4]);
  if (DIM == 3) {
    get4(a.u[C], R(y, zp), x0, nx, 0, S[5]);
    get4(a.u[C], R(y, zm), x0, nx, 0, S[6]);
  }
  // for every other axis A: u_A at +e_A, at +e_A - e_C, at the face, at -e_C
  T Up[DIM][4], Ux[DIM][4], U0[DIM][4], Um[DIM][4];
#pragma unroll
  for (int A = 0; A < DIM; ++A) {
    if (A == C) continue;
    const T *uA = a.u[A];
    if (A == 0) get4(uA, ro, x0, nx, 1, Up[A]);
    else if (A == 1) get4(uA, R(yp, z), x0, nx, 0, Up[A]);
    else get4(uA, R(y, zp), x0, nx, 0, Up[A]);
    int yy = y, zz = z, sh = 0;
    if (A == 0) sh = 1; else if (A == 1) yy = yp; else zz = zp;
    if (C == 0) sh -= 1; else if (C == 1) yy = ym; else zz = zm;
    get4(uA, R(yy, zz), x0, nx, sh, Ux[A]);
    get4(uA, ro, x0, nx, 0, U0[A]);
    if (C == 0) get4(uA, ro, x0, nx, -1, Um[A]);
    else if (C == 1) get4(uA, R(ym, z), x0, nx, 0, Um[A]);
    else get4(uA, R(y, zm), x0, nx, 0, Um[A]);
  }
  T nold[4], P0[4], Pm[4];
  if (!a.first) {
    T t0[4], t1[4];
    ld4(a.Nold[C] + ro + x0, nold);
    get4(a.p, ro, x0, nx, 0, t0);
    if (a.psi) get4(a.psi, ro, x0, nx, 0, t1);
    else t1[0] = t1[1] = t1[2] = t1[3] = T(0);
#pragma unroll
    for (int e = 0; e < 4; ++e) P0[e] = t0[e] + t1[e];
    const int rm = C == 0 ? ro : (C == 1 ? R(ym, z) : R(y, zm));
    get4(a.p, rm, x0, nx, C == 0 ? -1 : 0, t0);
    if (a.psi) get4(a.psi, rm, x0, nx, C == 0 ? -1 : 0, t1);
    else t1[0] = t1[1] = t1[2] = t1[3] = T(0);
#pragma unroll
    for (int e = 0; e < 4; ++e) Pm[e] = t0[e] + t1[e];
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) nold[e] = P0[e] = Pm[e] = T(0);
  }
  // the arithmetic of k_rhs
  T q4[DIM], s2 = T(0);
#pragma unroll
  for (int ax = 0; ax < DIM; ++ax) {
    q4[ax] = T(0.25) * a.inv_h[ax];
    s2 += a.inv_h2[ax];
  }
  T Rv[4], Nn[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const T u0 = S[0][e];
    T lap = T(-2) * s2 * u0, adv = T(0);
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
      const T up = S[1 + 2 * ax][e], um = S[2 + 2 * ax][e];
      lap = fma(up + um, a.inv_h2[ax], lap);
      T sp, sm;
      if (ax == C) {
        sp = u0 + up;
        sm = um + u0;
      } else {
        sp = Up[ax][e] + Ux[ax][e];
        sm = U0[ax][e] + Um[ax][e];
      }
      adv = fma(q4[ax], sp * up - sm * um, adv);
    }
    T acc = a.cmu * lap;
    acc = fma(a.ncg[C], P0[e] - Pm[e], acc);
    acc = fma(a.ncA, adv, acc);
    Rv[e] = fma(a.cN, nold[e], acc);
    Nn[e] = adv;
  }
  st4(a.scr[C] + ro + x0, Rv);
  st4(a.Nold[C] + ro + x0, Nn);
}

// The same right-hand side for n_x divisible by 4: a thread computes one
// component at 4 consecutive x cells from 128-bit row loads.  A CTA holds d
// warps, one per component, on the same 128 cells of an x line, so the rows
// the components share (the other components' velocities, p, psi) are fetched
// into the SM's L1 once for all of them; launch grid (n_x / 128, n_y, n_z).
// The arithmetic per cell is the one above.
template <typename T, int DIM>
__device__ __forceinline__ void rhs4_body(const RhsArgs<T> &a, const Blk &B) {
  const int x0 = 4 * (B.x * blockDim.x + threadIdx.x);
  const int y = B.y, z = B.z, c = threadIdx.y;
  if (x0 >= a.n[0]) return;
  if (c == 0) rhs4_component<T, DIM, 0>(a, x0, y, z);
  else if (c == 1) rhs4_component<T, DIM, 1>(a, x0, y, z);
  else if (DIM == 3) rhs4_component<T, DIM, DIM == 3 ? 2 : 1>(a, x0, y, z);
}
template <typename T, int DIM>
__global__ void __launch_bounds__(32 * DIM) k_rhs4(const RhsArgs<T> a) {
  pdl_wait();
  pdl_release();
  rhs4_body<T, DIM>(a, hw_blk());
}
template <typename T, int DIM>
__global__ void __launch_bounds__(32 * DIM) k_rhs4_b(const __grid_constant__ Batch<RhsArgs<T>> Bt) {
  pdl_wait();
  pdl_release();
  Blk b;
  const int i = batch_member(Bt, b);
  rhs4_body<T, DIM>(Bt.a[i], b);
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

// ---------------------------------------------------------------------------
// launchers

static inline unsigned grid_stride_blocks(long long work) {
  // 16 CTAs per SM at most, then grid-stride
  long long b = (work + 255) / 256;
  const long long sms = device_sms(), cap = (sms > 0 ? sms : 152) * 16;
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename T>
cudaError_t launch_rhs(int dim, const RhsArgs<T> &a, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {  // FP64 keeps the scalar kernel (register pressure)
    if ((a.n[0] & 3) == 0) {
      const dim3 blk(32, dim);
      const dim3 grid((unsigned)((a.n[0] / 4 + 31) / 32), (unsigned)a.n[1], (unsigned)(dim == 3 ? a.n[2] : 1));
      if (dim == 2) return launch_pdl(k_rhs4<T, 2>, grid, blk, 0, s, a);
      return launch_pdl(k_rhs4<T, 3>, grid, blk, 0, s, a);
    }
  }
  const long long cells = (long long)a.n[0] * a.n[1] * (dim == 3 ? a.n[2] : 1);
  const unsigned g = grid_stride_blocks(cells);
  if (dim == 2) return launch_pdl(k_rhs<T, 2>, dim3(g), dim3(256), 0, s, a);
  return launch_pdl(k_rhs<T, 3>, dim3(g), dim3(256), 0, s, a);
}

// all members share dim, precision and n (one ensemble size class)
template <typename T>
cudaError_t launch_rhs_batch(int dim, const RhsArgs<T> *a, int n, cudaStream_t s) {
  if (n < 1) return cudaSuccess;
  std::vector<dim3> g(n);
  if constexpr (sizeof(T) == 4) {
    if ((a[0].n[0] & 3) == 0) {
      for (int i = 0; i < n; ++i)
        g[i] = dim3((unsigned)((a[i].n[0] / 4 + 31) / 32), (unsigned)a[i].n[1], (unsigned)(dim == 3 ? a[i].n[2] : 1));
      if (dim == 2) return launch_batch(k_rhs4_b<T, 2>, a, g.data(), n, dim3(32, 2), s);
      return launch_batch(k_rhs4_b<T, 3>, a, g.data(), n, dim3(32, 3), s);
    }
  }
  for (int i = 0; i < n; ++i)
    g[i] = dim3(grid_stride_blocks((long long)a[i].n[0] * a[i].n[1] * (dim == 3 ? a[i].n[2] : 1)));
  if (dim == 2) return launch_batch(k_rhs_b<T, 2>, a, g.data(), n, dim3(256), s);
  return launch_batch(k_rhs_b<T, 3>, a, g.data(), n, dim3(256), s);
}
template cudaError_t launch_rhs_batch<float>(int, const RhsArgs<float> *, int, cudaStream_t);
template cudaError_t launch_rhs_batch<double>(int, const RhsArgs<double> *, int, cudaStream_t);

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
