// Batched constant-coefficient cyclic tridiagonal line solves (Sec. 4.2,
// eq. TriDiagX) for sm_103a.
//
// Every line system (1 + 2r) x_i - r x_{i-1} - r x_{i+1} = b_i (indices mod n)
// is solved through the exact factorisation
//     A = c (I - lam S)(I - lam S^{-1}),   lam = 2r / (1 + 2r + sqrt(1 + 4r)),
// S the cyclic shift and c = r / lam.  Each factor is a first-order cyclic
// recurrence y_i = lam y_{i-1} + b_i.  A line is cut into chunks; every chunk
// runs the recurrence locally from zero (the paper's local Thomas step on B_p,
// eq. LocalTriSystem), the chunk end values are combined by a scan across
// chunks (the interface system, eq. SchurSystem, which for a bidiagonal factor
// is a first-order recurrence over the chunks), and every element gets one
// correction term lam^(k) * carry (eq. SchurCorrection).  The periodic wrap is
// the rank-one term lam^{i+1} z_{n-1} / (1 - lam^n) (Sherman-Morrison on the
// factor), folded into the same correction.
//
// Two data layouts:
//   * x lines (contiguous): one warp per line, lane l owns chunk l of every
//     round of 128 elements (4 contiguous elements per lane), loaded as
//     128-bit vectors; the chunk scan is a warp shuffle scan.
//   * y / z lines (strided): a CTA owns 32 consecutive x columns; warp w owns
//     elements [w*CH, (w+1)*CH) of each of the 32 lines; every load
//     instruction of a warp reads 32 consecutive x values; the chunk scan runs
//     through shared memory.
// Each element is read once and written once: 2 words of HBM traffic.
#pragma once

#include "ib_internal.cuh"

namespace ibg {

#define IBG_FULL 0xffffffffu

template <typename T>
__device__ __forceinline__ T ld_ro(const T *p) { return __ldg(p); }

__device__ __forceinline__ int next_wrap(int i, int n) { return i + 1 == n ? 0 : i + 1; }

// D.u at cell (i, j, k): sum_a (u_a at face i_a + 1 - u_a at face i_a) / h_a
template <typename T>
__device__ __forceinline__ T div_at(const SweepArgs<T> &a, int i, int j, int k) {
  const int nx = a.n[0], ny = a.n[1];
  const long long o = i + (long long)nx * (j + (long long)ny * k);
  T d = (ld_ro(a.u[0] + (o - i + next_wrap(i, nx))) - ld_ro(a.u[0] + o)) * a.inv_h[0];
  d += (ld_ro(a.u[1] + (o + (long long)nx * (next_wrap(j, ny) - j))) - ld_ro(a.u[1] + o)) * a.inv_h[1];
  if (a.dim == 3)
    d += (ld_ro(a.u[2] + (o + (long long)nx * ny * (next_wrap(k, a.n[2]) - k))) - ld_ro(a.u[2] + o)) *
         a.inv_h[2];
  return d;
}

// right-hand side of one element
template <typename T, int PRO>
__device__ __forceinline__ T sweep_in(const SweepArgs<T> &a, const T *F, long long o, int i, int j, int k) {
  if (PRO == PRO_LOAD) return F[o];
  // Step 3e right-hand side -rho/dt D.u^{n+1}; D.u^{n+1} is kept for the next
  // step and the pressure takes the -chi mu D.(u^{n+1} + u^n)/2 part of Step 3f
  const T dn = div_at(a, i, j, k);
  const T dold = a.div[o];
  a.div[o] = dn;
  a.p[o] = a.p[o] - a.chi_mu_half * (dn + dold);
  return a.pro_scale * dn;
}

template <typename T, int EPI>
__device__ __forceinline__ void sweep_out(const SweepArgs<T> &a, T *F, int comp, long long o, T x) {
  if (EPI == EPI_STORE) {
    F[o] = x;
  } else if (EPI == EPI_ADDU) {  // u^{n+1} = u^n + e; the scratch starts the next step at zero
    a.uo[comp][o] += x;
    F[o] = T(0);
  } else {                       // psi^{n+1/2}; p += psi (Step 3f)
    F[o] = x;
    a.p[o] += x;
  }
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

// Solve one x line held by a warp: v[r][e] is element (32 r + lane) * 4 + e.
template <typename T, int R>
__device__ __forceinline__ void solve_line_warp(const LineCoef<T> &co, int n, int lane, T (&v)[R][4]) {
  const T lam = co.lam;
  const T *pw = co.pw;
  T cin[R];
  // forward factor (I - lam S) y = b
  T carry = T(0);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i0 = (r * 32 + lane) * 4;
    const int len = max(0, min(4, n - i0));
    T z = T(0);
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (e < len) { z = fma(lam, z, v[r][e]); v[r][e] = z; }
    T s = z, g = ld_ro(pw + len);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const T su = __shfl_up_sync(IBG_FULL, s, off);
      const T gu = __shfl_up_sync(IBG_FULL, g, off);
      if (lane >= off) { s = fma(su, g, s); g = gu * g; }
    }
    const T S = fma(g, carry, s);
    const T Sx = __shfl_up_sync(IBG_FULL, S, 1);
    cin[r] = lane == 0 ? carry : Sx;
    carry = __shfl_sync(IBG_FULL, S, 31);
  }
  T K = carry * co.inv_1m;  // periodic wrap: y_{-1} = z_{n-1} / (1 - lam^n)
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i0 = (r * 32 + lane) * 4;
    const int len = max(0, min(4, n - i0));
    const T t = fma(ld_ro(pw + min(i0, n)), K, cin[r]);
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (e < len) v[r][e] = fma(ld_ro(pw + e + 1), t, v[r][e]);
  }
  // backward factor (I - lam S^{-1}) x = y
  carry = T(0);
#pragma unroll
  for (int r = R - 1; r >= 0; --r) {
    const int i0 = (r * 32 + lane) * 4;
    const int len = max(0, min(4, n - i0));
    T z = T(0);
#pragma unroll
    for (int e = 3; e >= 0; --e)
      if (e < len) { z = fma(lam, z, v[r][e]); v[r][e] = z; }
    T s = z, g = ld_ro(pw + len);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const T sd = __shfl_down_sync(IBG_FULL, s, off);
      const T gd = __shfl_down_sync(IBG_FULL, g, off);
      if (lane + off < 32) { s = fma(sd, g, s); g = gd * g; }
    }
    const T S = fma(g, carry, s);
    const T Sx = __shfl_down_sync(IBG_FULL, S, 1);
    cin[r] = lane == 31 ? carry : Sx;
    carry = __shfl_sync(IBG_FULL, S, 0);
  }
  K = carry * co.inv_1m;  // x_n = x_0 = w_0 / (1 - lam^n)
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i0 = (r * 32 + lane) * 4;
    const int len = max(0, min(4, n - i0));
    if (len > 0) {
      const T t = fma(ld_ro(pw + (n - i0 - len)), K, cin[r]);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (e < len) v[r][e] = fma(ld_ro(pw + (len - e)), t, v[r][e]) * co.inv_c;
    }
  }
}

// one warp per x line; blockIdx.y selects the field
template <typename T, int R, int PRO, int EPI>
__global__ void __launch_bounds__(256) k_sweep_x(const SweepArgs<T> a) {
  const int lane = threadIdx.x & 31;
  const int nx = a.n[0], ny = a.n[1];
  const long long nlines = (long long)ny * (a.dim == 3 ? a.n[2] : 1);
  const long long line = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (line >= nlines) return;  // uniform per warp
  const int comp = blockIdx.y;
  T *F = a.f[comp];
  const T *Fin = a.fin[comp] ? a.fin[comp] : F;
  const int j = (int)(line % ny), k = (int)(line / ny);
  const long long base = line * nx;
  const bool vec = (nx & 3) == 0;
  T v[R][4];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i0 = (r * 32 + lane) * 4;
    if (PRO == PRO_LOAD && vec) {
      if (i0 < nx) ld4(Fin + base + i0, v[r]);
      else { v[r][0] = v[r][1] = v[r][2] = v[r][3] = T(0); }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = i0 + e;
        v[r][e] = i < nx ? sweep_in<T, PRO>(a, Fin, base + i, i, j, k) : T(0);
      }
    }
  }
  solve_line_warp<T, R>(a.co, nx, lane, v);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i0 = (r * 32 + lane) * 4;
    if (EPI == EPI_STORE && vec) {
      if (i0 < nx) st4(F + base + i0, v[r]);
    } else if (EPI == EPI_ADDU && vec) {
      if (i0 < nx) {
        T uu[4];
        ld4(a.uo[comp] + base + i0, uu);
#pragma unroll
        for (int e = 0; e < 4; ++e) uu[e] += v[r][e];
        st4(a.uo[comp] + base + i0, uu);
        const T zero[4] = {T(0), T(0), T(0), T(0)};
        st4(F + base + i0, zero);
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (i0 + e < nx) sweep_out<T, EPI>(a, F, comp, base + i0 + e, v[r][e]);
    }
  }
}

// strided lines along axis 1 (y) or 2 (z); blockIdx.x: 32 x columns,
// blockIdx.y: the remaining coordinate, blockIdx.z: the field
template <typename T, int CH, int W, int PRO, int EPI>
__global__ void __launch_bounds__(32 * W) k_sweep_s(const SweepArgs<T> a, const int axis) {
  __shared__ T sz[W][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nx = a.n[0], ny = a.n[1];
  const int x = blockIdx.x * 32 + lane;
  const int other = blockIdx.y;
  const int comp = blockIdx.z;
  T *F = a.f[comp];
  const T *Fin = a.fin[comp] ? a.fin[comp] : F;
  const int nl = a.n[axis];
  const long long stride = axis == 1 ? (long long)nx : (long long)nx * ny;
  const long long base = axis == 1 ? x + (long long)nx * ny * other : x + (long long)nx * other;
  const bool xok = x < nx;
  const int start = w * CH;
  const int len = max(0, min(CH, nl - start));
  const T lam = a.co.lam;
  const T *pw = a.co.pw;
  T v[CH];
#pragma unroll
  for (int e = 0; e < CH; ++e) {
    v[e] = T(0);
    if (xok && e < len) {
      const int t = start + e;
      v[e] = sweep_in<T, PRO>(a, Fin, base + t * stride, x, axis == 1 ? t : other, axis == 1 ? other : t);
    }
  }
  // forward factor
  T z = T(0);
#pragma unroll
  for (int e = 0; e < CH; ++e)
    if (e < len) { z = fma(lam, z, v[e]); v[e] = z; }
  sz[w][lane] = z;
  __syncthreads();
  T cin = T(0);
  for (int q = 0; q < w; ++q) cin = fma(cin, ld_ro(pw + max(0, min(CH, nl - q * CH))), sz[q][lane]);
  T tot = cin;
  for (int q = w; q < W; ++q) tot = fma(tot, ld_ro(pw + max(0, min(CH, nl - q * CH))), sz[q][lane]);
  T t = fma(ld_ro(pw + min(start, nl)), tot * a.co.inv_1m, cin);
#pragma unroll
  for (int e = 0; e < CH; ++e)
    if (e < len) v[e] = fma(ld_ro(pw + e + 1), t, v[e]);
  __syncthreads();
  // backward factor
  z = T(0);
#pragma unroll
  for (int e = CH - 1; e >= 0; --e)
    if (e < len) { z = fma(lam, z, v[e]); v[e] = z; }
  sz[w][lane] = z;
  __syncthreads();
  cin = T(0);
  for (int q = W - 1; q > w; --q) cin = fma(cin, ld_ro(pw + max(0, min(CH, nl - q * CH))), sz[q][lane]);
  tot = cin;
  for (int q = w; q >= 0; --q) tot = fma(tot, ld_ro(pw + max(0, min(CH, nl - q * CH))), sz[q][lane]);
  if (len > 0) {
    t = fma(ld_ro(pw + (nl - start - len)), tot * a.co.inv_1m, cin);
#pragma unroll
    for (int e = 0; e < CH; ++e)
      if (e < len) v[e] = fma(ld_ro(pw + (len - e)), t, v[e]) * a.co.inv_c;
  }
  if (xok) {
#pragma unroll
    for (int e = 0; e < CH; ++e)
      if (e < len) sweep_out<T, EPI>(a, F, comp, base + (start + e) * stride, v[e]);
  }
}

// line lengths 8 <= n <= 512 (checked by the caller)
template <typename T, int PRO, int EPI>
cudaError_t launch_sweep_t(int axis, int nfields, const SweepArgs<T> &a, cudaStream_t s) {
  const int nl = a.n[axis];
  if (axis == 0) {
    const long long nlines = (long long)a.n[1] * (a.dim == 3 ? a.n[2] : 1);
    dim3 grid((unsigned)((nlines + 7) / 8), nfields);
    if (nl <= 128) k_sweep_x<T, 1, PRO, EPI><<<grid, 256, 0, s>>>(a);
    else if (nl <= 256) k_sweep_x<T, 2, PRO, EPI><<<grid, 256, 0, s>>>(a);
    else k_sweep_x<T, 4, PRO, EPI><<<grid, 256, 0, s>>>(a);
  } else {
    const int other = axis == 1 ? (a.dim == 3 ? a.n[2] : 1) : a.n[1];
    dim3 grid((unsigned)((a.n[0] + 31) / 32), other, nfields);
    if (nl <= 64) k_sweep_s<T, 8, 8, PRO, EPI><<<grid, 256, 0, s>>>(a, axis);
    else if (nl <= 128) k_sweep_s<T, 16, 8, PRO, EPI><<<grid, 256, 0, s>>>(a, axis);
    else if (nl <= 256) k_sweep_s<T, 16, 16, PRO, EPI><<<grid, 512, 0, s>>>(a, axis);
    else k_sweep_s<T, 32, 16, PRO, EPI><<<grid, 512, 0, s>>>(a, axis);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sweep_impl(int axis, int pro, int epi, int nfields, const SweepArgs<T> &a, cudaStream_t s) {
  if (pro == PRO_LOAD && epi == EPI_STORE) return launch_sweep_t<T, PRO_LOAD, EPI_STORE>(axis, nfields, a, s);
  if (pro == PRO_LOAD && epi == EPI_ADDU) return launch_sweep_t<T, PRO_LOAD, EPI_ADDU>(axis, nfields, a, s);
  if (pro == PRO_DIV && epi == EPI_STORE) return launch_sweep_t<T, PRO_DIV, EPI_STORE>(axis, nfields, a, s);
  if (pro == PRO_LOAD && epi == EPI_P) return launch_sweep_t<T, PRO_LOAD, EPI_P>(axis, nfields, a, s);
  return cudaErrorInvalidValue;
}

}  // namespace ibg
