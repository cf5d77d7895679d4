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
// (loads only)
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

// Prologue of the first psi sweep (Step 3e right-hand side -rho/dt D.u^{n+1},
// and the -chi mu D.(u^{n+1} + u^n)/2 part of Step 3f): returns the
// right-hand side and the new div and p values, which the caller stores after
// all loads of the line have been issued.
template <typename T>
__device__ __forceinline__ T div_prologue(const SweepArgs<T> &a, long long o, int i, int j, int k, T &dnew,
                                          T &pnew) {
  dnew = div_at(a, i, j, k);
  pnew = a.p[o] - a.chi_mu_half * (dnew + a.div[o]);
  return a.pro_scale * dnew;
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

// The same solve when n == 128 R: every lane chunk holds exactly 4 elements,
// so every chunk's gain is lam^4 and a window of 2^k chunks has gain
// lam^(4 2^k); the scan then shuffles only the partial sums and all powers
// live in registers.
template <typename T, int R>
__device__ __forceinline__ void solve_line_warp_full(const LineCoef<T> &co, int n, int lane, T (&v)[R][4]) {
  const T lam = co.lam;
  const T *pw = co.pw;
  const T l1 = lam, l2 = ld_ro(pw + 2), l3 = ld_ro(pw + 3), l4 = ld_ro(pw + 4);
  T gk[5];  // lam^(4 * 2^k), k = 0..4
#pragma unroll
  for (int q = 0; q < 5; ++q) gk[q] = ld_ro(pw + (4 << q));
  const T glane_f = ld_ro(pw + 4 * (lane + 1));   // gain of lanes 0..lane
  const T glane_b = ld_ro(pw + 4 * (32 - lane));  // gain of lanes lane..31
  T cin[R];
  // forward factor
  T carry = T(0);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    T z = v[r][0];
    v[r][1] = z = fma(lam, z, v[r][1]);
    v[r][2] = z = fma(lam, z, v[r][2]);
    v[r][3] = z = fma(lam, z, v[r][3]);
    T s = z;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const T su = __shfl_up_sync(IBG_FULL, s, 1 << q);
      if (lane >= (1 << q)) s = fma(su, gk[q], s);
    }
    const T S = fma(glane_f, carry, s);
    const T Sx = __shfl_up_sync(IBG_FULL, S, 1);
    cin[r] = lane == 0 ? carry : Sx;
    carry = __shfl_sync(IBG_FULL, S, 31);
  }
  T K = carry * co.inv_1m;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const T t = fma(ld_ro(pw + (r * 32 + lane) * 4), K, cin[r]);
    v[r][0] = fma(l1, t, v[r][0]);
    v[r][1] = fma(l2, t, v[r][1]);
    v[r][2] = fma(l3, t, v[r][2]);
    v[r][3] = fma(l4, t, v[r][3]);
  }
  // backward factor
  carry = T(0);
#pragma unroll
  for (int r = R - 1; r >= 0; --r) {
    T z = v[r][3];
    v[r][2] = z = fma(lam, z, v[r][2]);
    v[r][1] = z = fma(lam, z, v[r][1]);
    v[r][0] = z = fma(lam, z, v[r][0]);
    T s = z;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const T sd = __shfl_down_sync(IBG_FULL, s, 1 << q);
      if (lane + (1 << q) < 32) s = fma(sd, gk[q], s);
    }
    const T S = fma(glane_b, carry, s);
    const T Sx = __shfl_down_sync(IBG_FULL, S, 1);
    cin[r] = lane == 31 ? carry : Sx;
    carry = __shfl_sync(IBG_FULL, S, 0);
  }
  K = carry * co.inv_1m;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const T t = fma(ld_ro(pw + (n - (r * 32 + lane) * 4 - 4)), K, cin[r]);
    v[r][0] = fma(l4, t, v[r][0]) * co.inv_c;
    v[r][1] = fma(l3, t, v[r][1]) * co.inv_c;
    v[r][2] = fma(l2, t, v[r][2]) * co.inv_c;
    v[r][3] = fma(l1, t, v[r][3]) * co.inv_c;
  }
}

// one warp per x line; blockIdx.y selects the field
template <typename T, int R, int PRO, int EPI, bool FULL>
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
  T dn[PRO == PRO_DIV ? R : 1][4], pn[PRO == PRO_DIV ? R : 1][4];
  // loads (no stores until every load of the line is issued)
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i0 = (r * 32 + lane) * 4;
    if (PRO == PRO_LOAD && vec) {
      if (i0 < nx) ld4(Fin + base + i0, v[r]);
      else { v[r][0] = v[r][1] = v[r][2] = v[r][3] = T(0); }
    } else if (PRO == PRO_DIV && vec) {
      T u4[4], vj[4], vj1[4], d4[4], p4[4];
      const T *u0 = a.u[0], *u1 = a.u[1];
      if (i0 < nx) {
        ld4(u0 + base + i0, u4);
        ld4(u1 + base + i0, vj);
        ld4(u1 + base + (long long)nx * (next_wrap(j, ny) - j) + i0, vj1);
        ld4(a.div + base + i0, d4);
        ld4(a.p + base + i0, p4);
      }
      // u at face i0 + 4: the next lane's first element, or a load at the end
      // of a round / the periodic wrap at the end of the line
      const T nb = __shfl_down_sync(IBG_FULL, u4[0], 1);
      T unext = nb;
      if (i0 < nx && (lane == 31 || i0 + 4 >= nx)) unext = ld_ro(u0 + base + (i0 + 4 < nx ? i0 + 4 : 0));
      T w4[4] = {T(0), T(0), T(0), T(0)}, wk1[4] = {T(0), T(0), T(0), T(0)};
      if (a.dim == 3 && i0 < nx) {
        ld4(a.u[2] + base + i0, w4);
        ld4(a.u[2] + base + (long long)nx * ny * (next_wrap(k, a.n[2]) - k) + i0, wk1);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const T up = e < 3 ? u4[e + 1] : unext;
        T d = (up - u4[e]) * a.inv_h[0];
        d += (vj1[e] - vj[e]) * a.inv_h[1];
        if (a.dim == 3) d += (wk1[e] - w4[e]) * a.inv_h[2];
        dn[PRO == PRO_DIV ? r : 0][e] = d;
        pn[PRO == PRO_DIV ? r : 0][e] = p4[e] - a.chi_mu_half * (d + d4[e]);
        v[r][e] = i0 < nx ? a.pro_scale * d : T(0);
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = i0 + e;
        if (PRO == PRO_DIV) {
          v[r][e] = i < nx ? div_prologue<T>(a, base + i, i, j, k, dn[PRO == PRO_DIV ? r : 0][e],
                                             pn[PRO == PRO_DIV ? r : 0][e])
                           : T(0);
        } else {
          v[r][e] = i < nx ? Fin[base + i] : T(0);
        }
      }
    }
  }
  if (PRO == PRO_DIV) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i0 = (r * 32 + lane) * 4;
      if (vec) {
        if (i0 < nx) {
          st4(a.div + base + i0, dn[PRO == PRO_DIV ? r : 0]);
          st4(a.p + base + i0, pn[PRO == PRO_DIV ? r : 0]);
        }
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (i0 + e < nx) {
            a.div[base + i0 + e] = dn[PRO == PRO_DIV ? r : 0][e];
            a.p[base + i0 + e] = pn[PRO == PRO_DIV ? r : 0][e];
          }
      }
    }
  }
  if (FULL) solve_line_warp_full<T, R>(a.co, nx, lane, v);
  else solve_line_warp<T, R>(a.co, nx, lane, v);
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
    } else if (EPI == EPI_P && vec) {
      if (i0 < nx) {
        T pp[4];
        ld4(a.p + base + i0, pp);
#pragma unroll
        for (int e = 0; e < 4; ++e) pp[e] += v[r][e];
        st4(F + base + i0, v[r]);
        st4(a.p + base + i0, pp);
      }
    } else {
      T old[4] = {T(0), T(0), T(0), T(0)};
      if (EPI != EPI_STORE) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (i0 + e < nx) old[e] = EPI == EPI_ADDU ? a.uo[comp][base + i0 + e] : a.p[base + i0 + e];
      }
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (i0 + e < nx) {
          const long long o = base + i0 + e;
          if (EPI == EPI_STORE) {
            F[o] = v[r][e];
          } else if (EPI == EPI_ADDU) {
            a.uo[comp][o] = old[e] + v[r][e];
            F[o] = T(0);
          } else {
            F[o] = v[r][e];
            a.p[o] = old[e] + v[r][e];
          }
        }
    }
  }
}

// strided lines along axis 1 (y) or 2 (z); blockIdx.x: 32 x columns,
// blockIdx.y: the remaining coordinate, blockIdx.z: the field.  FULL: the
// line length is exactly W * CH, so no element needs a bounds test.
// Element offsets fit in 32 bits (at most 512^3 elements per field).
template <typename T, int CH, int W, int PRO, int EPI, bool FULL>
__global__ void __launch_bounds__(32 * W) k_sweep_s(const SweepArgs<T> a, const int axis) {
  __shared__ T sz[W][33];
  __shared__ T lp[CH + 1];  // lam^0 .. lam^CH
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nx = a.n[0], ny = a.n[1];
  const int x = blockIdx.x * 32 + lane;
  const int other = blockIdx.y;
  if (threadIdx.x <= CH) lp[threadIdx.x] = ld_ro(a.co.pw + threadIdx.x);
  const int comp = blockIdx.z;
  T *F = a.f[comp];
  const T *Fin = a.fin[comp] ? a.fin[comp] : F;
  const int nl = a.n[axis];
  const int stride = axis == 1 ? nx : nx * ny;
  const int base = axis == 1 ? x + nx * ny * other : x + nx * other;
  const bool xok = x < nx;
  const int start = w * CH;
  const int len = FULL ? CH : max(0, min(CH, nl - start));
  const T lam = a.co.lam;
  const T *pw = a.co.pw;
  const int o0 = base + start * stride;
  T v[CH];
  T pn[PRO == PRO_DIV ? CH : 1];
  if (PRO == PRO_LOAD) {
#pragma unroll
    for (int e = 0; e < CH; ++e) v[e] = (xok && (FULL || e < len)) ? Fin[o0 + e * stride] : T(0);
  } else {
    // Step 3e right-hand side -rho/dt D.u^{n+1}; the new D.u and p are stored
    // after every load of the chunk (see below)
    const int dx = x + 1 == nx ? 1 - nx : 1;
    const int nz = a.dim == 3 ? a.n[2] : 1;
    const int jo = axis == 1 ? -1 : other, ko = axis == 1 ? other : -1;  // fixed coordinate
    const int ld_y = nx, ld_z = nx * ny;
#pragma unroll
    for (int e = 0; e < CH; ++e) {
      v[e] = T(0);
      pn[PRO == PRO_DIV ? e : 0] = T(0);
      if (xok && (FULL || e < len)) {
        const int t = start + e;
        const int j = axis == 1 ? t : jo, k = axis == 1 ? ko : t;
        const int o = o0 + e * stride;
        const int dy = j + 1 == ny ? ld_y * (1 - ny) : ld_y;
        T d = (ld_ro(a.u[0] + o + dx) - ld_ro(a.u[0] + o)) * a.inv_h[0];
        d += (ld_ro(a.u[1] + o + dy) - ld_ro(a.u[1] + o)) * a.inv_h[1];
        if (a.dim == 3) {
          const int dz = k + 1 == nz ? ld_z * (1 - nz) : ld_z;
          d += (ld_ro(a.u[2] + o + dz) - ld_ro(a.u[2] + o)) * a.inv_h[2];
        }
        pn[PRO == PRO_DIV ? e : 0] = a.p[o] - a.chi_mu_half * (d + a.div[o]);
        v[e] = a.pro_scale * d;
      }
    }
    if (xok) {
      const T inv_scale = T(1) / a.pro_scale;
#pragma unroll
      for (int e = 0; e < CH; ++e)
        if (FULL || e < len) {
          const int o = o0 + e * stride;
          a.div[o] = v[e] * inv_scale;
          a.p[o] = pn[PRO == PRO_DIV ? e : 0];
        }
    }
  }
  // forward factor (I - lam S) y = b: local pass, chunk scan, correction
  T z = T(0);
#pragma unroll
  for (int e = 0; e < CH; ++e)
    if (FULL || e < len) { z = fma(lam, z, v[e]); v[e] = z; }
  sz[w][lane] = z;
  __syncthreads();
  T cin = T(0);
  for (int q = 0; q < w; ++q) cin = fma(cin, FULL ? lp[CH] : ld_ro(pw + max(0, min(CH, nl - q * CH))), sz[q][lane]);
  T tot = cin;
  for (int q = w; q < W; ++q) tot = fma(tot, FULL ? lp[CH] : ld_ro(pw + max(0, min(CH, nl - q * CH))), sz[q][lane]);
  T t = fma(ld_ro(pw + min(start, nl)), tot * a.co.inv_1m, cin);
#pragma unroll
  for (int e = 0; e < CH; ++e)
    if (FULL || e < len) v[e] = fma(lp[e + 1], t, v[e]);
  __syncthreads();
  // backward factor (I - lam S^{-1}) x = y
  z = T(0);
#pragma unroll
  for (int e = CH - 1; e >= 0; --e)
    if (FULL || e < len) { z = fma(lam, z, v[e]); v[e] = z; }
  sz[w][lane] = z;
  __syncthreads();
  cin = T(0);
  for (int q = W - 1; q > w; --q) cin = fma(cin, FULL ? lp[CH] : ld_ro(pw + max(0, min(CH, nl - q * CH))), sz[q][lane]);
  tot = cin;
  for (int q = w; q >= 0; --q) tot = fma(tot, FULL ? lp[CH] : ld_ro(pw + max(0, min(CH, nl - q * CH))), sz[q][lane]);
  if (FULL || len > 0) {
    t = fma(ld_ro(pw + (nl - start - len)), tot * a.co.inv_1m, cin);
#pragma unroll
    for (int e = 0; e < CH; ++e)
      if (FULL || e < len) {
        const int pe = FULL ? CH - e : max(0, len - e);
        v[e] = fma(lp[pe], t, v[e]) * a.co.inv_c;
      }
  }
  if (!xok) return;
  if (EPI == EPI_STORE) {
#pragma unroll
    for (int e = 0; e < CH; ++e)
      if (FULL || e < len) F[o0 + e * stride] = v[e];
  } else {
    // scratch / psi stores first, then every load of the old values, then the
    // sums: no load waits behind a store
    T *tgt = EPI == EPI_ADDU ? a.uo[comp] : a.p;
#pragma unroll
    for (int e = 0; e < CH; ++e)
      if (FULL || e < len) F[o0 + e * stride] = EPI == EPI_ADDU ? T(0) : v[e];  // clear scratch / store psi
#pragma unroll
    for (int e = 0; e < CH; ++e)
      if (FULL || e < len) v[e] += tgt[o0 + e * stride];
#pragma unroll
    for (int e = 0; e < CH; ++e)
      if (FULL || e < len) tgt[o0 + e * stride] = v[e];
  }
}

// line lengths 8 <= n <= 512 (checked by the caller)
template <typename T, int PRO, int EPI>
cudaError_t launch_sweep_t(int axis, int nfields, const SweepArgs<T> &a, cudaStream_t s) {
  const int nl = a.n[axis];
  if (axis == 0) {
    const long long nlines = (long long)a.n[1] * (a.dim == 3 ? a.n[2] : 1);
    dim3 grid((unsigned)((nlines + 7) / 8), nfields);
    if (nl == 128) k_sweep_x<T, 1, PRO, EPI, true><<<grid, 256, 0, s>>>(a);
    else if (nl < 128) k_sweep_x<T, 1, PRO, EPI, false><<<grid, 256, 0, s>>>(a);
    else if (nl == 256) k_sweep_x<T, 2, PRO, EPI, true><<<grid, 256, 0, s>>>(a);
    else if (nl < 256) k_sweep_x<T, 2, PRO, EPI, false><<<grid, 256, 0, s>>>(a);
    else if (nl == 512) k_sweep_x<T, 4, PRO, EPI, true><<<grid, 256, 0, s>>>(a);
    else k_sweep_x<T, 4, PRO, EPI, false><<<grid, 256, 0, s>>>(a);
  } else {
    const int other = axis == 1 ? (a.dim == 3 ? a.n[2] : 1) : a.n[1];
    dim3 grid((unsigned)((a.n[0] + 31) / 32), other, nfields);
    if (nl == 64) k_sweep_s<T, 8, 8, PRO, EPI, true><<<grid, 256, 0, s>>>(a, axis);
    else if (nl < 64) k_sweep_s<T, 8, 8, PRO, EPI, false><<<grid, 256, 0, s>>>(a, axis);
    else if (nl == 128) k_sweep_s<T, 16, 8, PRO, EPI, true><<<grid, 256, 0, s>>>(a, axis);
    else if (nl < 128) k_sweep_s<T, 16, 8, PRO, EPI, false><<<grid, 256, 0, s>>>(a, axis);
    else if (nl == 256) k_sweep_s<T, 16, 16, PRO, EPI, true><<<grid, 512, 0, s>>>(a, axis);
    else if (nl < 256) k_sweep_s<T, 16, 16, PRO, EPI, false><<<grid, 512, 0, s>>>(a, axis);
    else if constexpr (sizeof(T) == 8) {  // FP64: fewer, longer chunks keep 512-thread CTAs within registers
      if (nl == 512) k_sweep_s<T, 32, 16, PRO, EPI, true><<<grid, 512, 0, s>>>(a, axis);
      else k_sweep_s<T, 32, 16, PRO, EPI, false><<<grid, 512, 0, s>>>(a, axis);
    } else if (nl == 512) k_sweep_s<T, 16, 32, PRO, EPI, true><<<grid, 1024, 0, s>>>(a, axis);
    else k_sweep_s<T, 16, 32, PRO, EPI, false><<<grid, 1024, 0, s>>>(a, axis);
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
