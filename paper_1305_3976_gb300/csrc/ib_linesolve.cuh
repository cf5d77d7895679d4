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

#include <vector>

#include "ib_internal.cuh"

namespace ibg {

#define IBG_FULL 0xffffffffu

template <typename T>
__device__ __forceinline__ T ld_ro(const T *p) { return __ldg(p); }
// 4 contiguous elements through the read-only path (alignment as ld4)
__device__ __forceinline__ void ld4_ro(const float *p, float (&v)[4]) {
  const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4_ro(const double *p, double (&v)[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
  const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

__device__ __forceinline__ int next_wrap(int i, int n) { return i + 1 == n ? 0 : i + 1; }

// dynamic shared memory of the strided sweeps: D.u^{n+1} of every element of
// the CTA between the divergence prologue and the update of p after the solve
// (sweep_s_div_smem bytes; none for the other sweeps)
extern __shared__ __align__(16) unsigned char ibg_sweep_dyn[];

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

// p^{n-1/2} as it enters p^{n+1/2}: itself (Step 3f), or nothing in the
// first-order variant (Sec. 3.1), whose solve gives the pressure directly
template <typename T>
__device__ __forceinline__ T kept_p(const SweepArgs<T> &a, T p) {
  return a.p_keep != T(0) ? a.p_keep * p : T(0);
}

// Prologue of the first psi sweep (Step 3e right-hand side -rho/dt D.u^{n+1},
// and the -chi mu D.(u^{n+1} + u^n)/2 part of Step 3f): returns the
// right-hand side and the new div and p values, which the caller stores after
// all loads of the line have been issued.
template <typename T>
__device__ __forceinline__ T div_prologue(const SweepArgs<T> &a, long long o, int i, int j, int k, T &dnew,
                                          T &pnew) {
  dnew = div_at(a, i, j, k);
  pnew = kept_p(a, a.p[o]) - a.chi_mu_half * (dnew + a.div[o]);
  return a.pro_scale * dnew;
}

// VW consecutive elements (VW = 1, 2, 4), VW-aligned
template <int VW, typename T>
__device__ __forceinline__ void ldv(const T *p, T (&v)[VW]) {
  if (VW == 4) {
    T t[4];
    ld4(p, t);
#pragma unroll
    for (int i = 0; i < VW; ++i) v[i] = t[i];
  } else if (VW == 2) {
    if (sizeof(T) == 4) {
      const float2 t = *reinterpret_cast<const float2 *>(p);
      v[0] = (T)t.x;
      v[VW - 1] = (T)t.y;
    } else {
      const double2 t = *reinterpret_cast<const double2 *>(p);
      v[0] = (T)t.x;
      v[VW - 1] = (T)t.y;
    }
  } else {
    v[0] = *p;
  }
}
// the same through the read-only path
template <int VW, typename T>
__device__ __forceinline__ void ldv_ro(const T *p, T (&v)[VW]) {
  if (VW == 4) {
    T t[4];
    ld4_ro(p, t);
#pragma unroll
    for (int i = 0; i < VW; ++i) v[i] = t[i];
  } else if (VW == 2) {
    if (sizeof(T) == 4) {
      const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
      v[0] = (T)t.x;
      v[VW - 1] = (T)t.y;
    } else {
      const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
      v[0] = (T)t.x;
      v[VW - 1] = (T)t.y;
    }
  } else {
    v[0] = __ldg(p);
  }
}
template <int VW, typename T>
__device__ __forceinline__ void stv(T *p, const T (&v)[VW]) {
  if (VW == 4) {
    T t[4] = {v[0], v[VW > 1 ? 1 : 0], v[VW > 2 ? 2 : 0], v[VW > 3 ? 3 : 0]};
    st4(p, t);
  } else if (VW == 2) {
    if (sizeof(T) == 4) *reinterpret_cast<float2 *>(p) = make_float2((float)v[0], (float)v[VW - 1]);
    else *reinterpret_cast<double2 *>(p) = make_double2((double)v[0], (double)v[VW - 1]);
  } else {
    *p = v[0];
  }
}

// Per-lane constants of a full-length x line (n = 128 R): loaded once per
// warp and reused for every line it solves.
template <typename T, int R>
struct XLineCoef {
  T lam, l2, l3, l4, inv_1m;
  T gk[5];      // lam^(4 * 2^k)
  T gf, gb;     // gains of lanes 0..lane and lane..31
  T pf[R], pb[R];  // lam^(i0) and lam^(n - i0 - 4) of this lane's chunks
  T inv_1m_lo;     // FP64-accurate periodic correction (EXT): the FP32 remainders
  const T *pw_lo;
  int n;
  __device__ __forceinline__ void load(const LineCoef<T> &co, int n_, int lane) {
    const int n = n_;
    this->n = n_;
    const T *pw = co.pw;
    lam = co.lam;
    inv_1m = co.inv_1m;
    inv_1m_lo = co.inv_1m_lo;
    pw_lo = co.pw_lo;
    l2 = ld_ro(pw + 2);
    l3 = ld_ro(pw + 3);
    l4 = ld_ro(pw + 4);
#pragma unroll
    for (int q = 0; q < 5; ++q) gk[q] = ld_ro(pw + (4 << q));
    gf = ld_ro(pw + 4 * (lane + 1));
    gb = ld_ro(pw + 4 * (32 - lane));
#pragma unroll
    for (int r = 0; r < R; ++r) {
      pf[r] = ld_ro(pw + (r * 32 + lane) * 4);
      pb[r] = ld_ro(pw + (n - (r * 32 + lane) * 4 - 4));
    }
  }
};

// Solve one x line held by a warp: v[r][e] is element (32 r + lane) * 4 + e.
template <typename T, int R, bool EXT>
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
  // periodic wrap: y_{-1} = z_{n-1} / (1 - lam^n)
  T tot = carry;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i0 = (r * 32 + lane) * 4;
    const int len = max(0, min(4, n - i0));
    const T t = wrap_term<EXT>(co, min(i0, n), tot, cin[r]);
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
  tot = carry;  // x_n = x_0 = w_0 / (1 - lam^n)
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i0 = (r * 32 + lane) * 4;
    const int len = max(0, min(4, n - i0));
    if (len > 0) {
      const T t = wrap_term<EXT>(co, n - i0 - len, tot, cin[r]);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (e < len) v[r][e] = fma(ld_ro(pw + (len - e)), t, v[r][e]);
    }
  }
}

// The same solve when n == 128 R: every lane chunk holds exactly 4 elements,
// so every chunk's gain is lam^4 and a window of 2^k chunks has gain
// lam^(4 2^k); the scan then shuffles only the partial sums and all powers
// live in registers.
template <typename T, int R, bool EXT>
__device__ __forceinline__ void solve_line_warp_full(const XLineCoef<T, R> &c, int lane, T (&v)[R][4]) {
  const T lam = c.lam;
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
      if (lane >= (1 << q)) s = fma(su, c.gk[q], s);
    }
    const T S = fma(c.gf, carry, s);
    const T Sx = __shfl_up_sync(IBG_FULL, S, 1);
    cin[r] = lane == 0 ? carry : Sx;
    carry = __shfl_sync(IBG_FULL, S, 31);
  }
  T K = carry * c.inv_1m;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const T t = EXT ? wrap_term_ext(c.pf[r], __ldg(c.pw_lo + (r * 32 + lane) * 4), c.inv_1m, c.inv_1m_lo, carry,
                                      cin[r])
                      : fma(c.pf[r], K, cin[r]);
    v[r][0] = fma(lam, t, v[r][0]);
    v[r][1] = fma(c.l2, t, v[r][1]);
    v[r][2] = fma(c.l3, t, v[r][2]);
    v[r][3] = fma(c.l4, t, v[r][3]);
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
      if (lane + (1 << q) < 32) s = fma(sd, c.gk[q], s);
    }
    const T S = fma(c.gb, carry, s);
    const T Sx = __shfl_down_sync(IBG_FULL, S, 1);
    cin[r] = lane == 31 ? carry : Sx;
    carry = __shfl_sync(IBG_FULL, S, 0);
  }
  K = carry * c.inv_1m;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const T t = EXT ? wrap_term_ext(c.pb[r], __ldg(c.pw_lo + (c.n - (r * 32 + lane) * 4 - 4)), c.inv_1m,
                                      c.inv_1m_lo, carry, cin[r])
                      : fma(c.pb[r], K, cin[r]);
    v[r][0] = fma(c.l4, t, v[r][0]);
    v[r][1] = fma(c.l3, t, v[r][1]);
    v[r][2] = fma(c.l2, t, v[r][2]);
    v[r][3] = fma(lam, t, v[r][3]);
  }
}

// one x line per warp and loop iteration; blockIdx.y selects the field
template <typename T, int R, int PRO, int EPI, bool FULL, bool EXT>
__device__ __forceinline__ void sweep_x_line(const SweepArgs<T> &a, const XLineCoef<T, R> &xc, T *F, const T *Fin,
                                             int comp, long long line, int lane) {
  const int nx = a.n[0], ny = a.n[1];
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
      // read-only loads (every element is read before this thread alone
      // writes it), and the new D.u and p stored at once: nothing of the
      // prologue stays live across the rounds
      T u4[4] = {T(0), T(0), T(0), T(0)}, vj[4] = {T(0), T(0), T(0), T(0)}, vj1[4] = {T(0), T(0), T(0), T(0)};
      T d4[4] = {T(0), T(0), T(0), T(0)}, p4[4] = {T(0), T(0), T(0), T(0)};
      const T *u0 = a.u[0], *u1 = a.u[1];
      if (i0 < nx) {
        ld4_ro(u0 + base + i0, u4);
        ld4_ro(u1 + base + i0, vj);
        ld4_ro(u1 + base + (long long)nx * (next_wrap(j, ny) - j) + i0, vj1);
        ld4_ro(a.div + base + i0, d4);
        ld4_ro(a.p + base + i0, p4);
      }
      // u at face i0 + 4: the next lane's first element, or a load at the end
      // of a round / the periodic wrap at the end of the line
      const T nb = __shfl_down_sync(IBG_FULL, u4[0], 1);
      T unext = nb;
      if (i0 < nx && (lane == 31 || i0 + 4 >= nx)) unext = ld_ro(u0 + base + (i0 + 4 < nx ? i0 + 4 : 0));
      T w4[4] = {T(0), T(0), T(0), T(0)}, wk1[4] = {T(0), T(0), T(0), T(0)};
      if (a.dim == 3 && i0 < nx) {
        ld4_ro(a.u[2] + base + i0, w4);
        ld4_ro(a.u[2] + base + (long long)nx * ny * (next_wrap(k, a.n[2]) - k) + i0, wk1);
      }
      T dn4[4], pn4[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const T up = e < 3 ? u4[e + 1] : unext;
        T d = (up - u4[e]) * a.inv_h[0];
        d += (vj1[e] - vj[e]) * a.inv_h[1];
        if (a.dim == 3) d += (wk1[e] - w4[e]) * a.inv_h[2];
        dn4[e] = d;
        pn4[e] = kept_p(a, p4[e]) - a.chi_mu_half * (d + d4[e]);
        v[r][e] = i0 < nx ? a.pro_scale * d : T(0);
      }
      if (i0 < nx) {
        st4(a.div + base + i0, dn4);
        st4(a.p + base + i0, pn4);
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
  // EARLY: the epilogue's old values (u^n or p) are loaded with the
  // right-hand sides, so their latency hides behind the solve
  constexpr bool EARLY = PRO == PRO_LOAD && EPI != EPI_STORE;
  T old4[EARLY ? R : 1][4];
  if (EARLY && vec) {
    const T *tgt = EPI == EPI_ADDU ? a.uo[comp] : a.p;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i0 = (r * 32 + lane) * 4;
      if (i0 < nx) ld4(tgt + base + i0, old4[EARLY ? r : 0]);
    }
  }
  if (PRO == PRO_DIV && !vec) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i0 = (r * 32 + lane) * 4;
      {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (i0 + e < nx) {
            a.div[base + i0 + e] = dn[PRO == PRO_DIV ? r : 0][e];
            a.p[base + i0 + e] = pn[PRO == PRO_DIV ? r : 0][e];
          }
      }
    }
  }
  if (FULL) solve_line_warp_full<T, R, EXT>(xc, lane, v);
  else solve_line_warp<T, R, EXT>(a.co, nx, lane, v);
  // the scale 1/c (EPI_ADDU folds it into the sum); skipped in the unscaled
  // sweeps of a chain
  const T sc = a.co.scale;
  if (EPI != EPI_ADDU && sc != T(1)) {
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int e = 0; e < 4; ++e) v[r][e] *= sc;
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i0 = (r * 32 + lane) * 4;
    if (EPI == EPI_STORE && vec) {
      if (i0 < nx) st4(F + base + i0, v[r]);
    } else if (EPI == EPI_ADDU && vec) {
      if (i0 < nx) {
        T uu[4];
        if (EARLY) {
#pragma unroll
          for (int e = 0; e < 4; ++e) uu[e] = old4[EARLY ? r : 0][e];
        } else {
          ld4(a.uo[comp] + base + i0, uu);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) uu[e] = fma(v[r][e], sc, uu[e]);
        st4(a.uo[comp] + base + i0, uu);
      }
    } else if (EPI == EPI_P && vec) {
      if (i0 < nx) {
        T pp[4];
        if (EARLY) {
#pragma unroll
          for (int e = 0; e < 4; ++e) pp[e] = old4[EARLY ? r : 0][e];
        } else {
          ld4(a.p + base + i0, pp);
        }
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
            a.uo[comp][o] = fma(v[r][e], sc, old[e]);
          } else {
            F[o] = v[r][e];
            a.p[o] = old[e] + v[r][e];
          }
        }
    }
  }
}

template <typename T, int R, int PRO, int EPI, bool FULL, bool EXT>
__device__ __forceinline__ void sweep_x_body(const SweepArgs<T> &a, const Blk &B) {
  const int lane = threadIdx.x & 31;
  const int nx = a.n[0], ny = a.n[1];
  const long long nlines = (long long)ny * (a.dim == 3 ? a.n[2] : 1);
  const int comp = B.y;
  T *F = a.f[comp];
  const T *Fin = a.fin[comp] ? a.fin[comp] : F;
  XLineCoef<T, R> xc;
  if (FULL) xc.load(a.co, nx, lane);
  // each warp solves lines warp, warp + W, ... (W warps in the grid)
  const long long wstride = (long long)B.gx * (blockDim.x >> 5);
  for (long long line = (long long)B.x * (blockDim.x >> 5) + (threadIdx.x >> 5); line < nlines; line += wstride)
    sweep_x_line<T, R, PRO, EPI, FULL, EXT>(a, xc, F, Fin, comp, line, lane);
}
template <typename T, int R, int PRO, int EPI, bool FULL, bool EXT>
__global__ void __launch_bounds__(256, PRO == PRO_DIV && R == 4 ? 3 : 1) k_sweep_x(const SweepArgs<T> a) {
  pdl_wait();
  pdl_release();
  sweep_x_body<T, R, PRO, EPI, FULL, EXT>(a, hw_blk());
}
template <typename T, int R, int PRO, int EPI, bool FULL, bool EXT>
__global__ void __launch_bounds__(256) k_sweep_x_b(const __grid_constant__ Batch<SweepArgs<T>> Bt) {
  pdl_wait();
  pdl_release();
  Blk b;
  const int i = batch_member(Bt, b);
  sweep_x_body<T, R, PRO, EPI, FULL, EXT>(Bt.a[i], b);
}

// strided lines along axis 1 (y) or 2 (z); a thread owns VW adjacent x
// columns (VW-wide vector loads, so a warp reads 32 VW consecutive values of
// a row); blockIdx.x: 32 VW x columns, blockIdx.y: the remaining coordinate,
// blockIdx.z: the field.  FULL: the line length is exactly W * CH, so no
// element needs a bounds test.  Element offsets fit in 32 bits (at most 512^3
// elements per field).
template <typename T, int VW, int CH, int W, int PRO, int EPI, bool FULL, bool EXT>
__device__ __forceinline__ void sweep_s_body(const SweepArgs<T> &a, const int axis, const Blk &B) {
  __shared__ T sz[W][VW][33];
  __shared__ T stot[VW][32];
  __shared__ T lp[CH + 1];  // lam^0 .. lam^CH
  // SCAN1 (FP64): warp 0 alone turns the chunk ends into the chunk prefixes
  // (W operations per column instead of W per column and warp), the same
  // operation sequence as every warp's own scan; FP32 keeps the per-warp scan
  constexpr bool SCAN1 = sizeof(T) == 8;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nx = a.n[0], ny = a.n[1];
  const int x0 = (B.x * 32 + lane) * VW;
  const int other = B.y;
  const int comp = B.z;
  if (threadIdx.x <= CH) lp[threadIdx.x] = ld_ro(a.co.pw + threadIdx.x);
  T *F = a.f[comp];
  const T *Fin = a.fin[comp] ? a.fin[comp] : F;
  const int nl = a.n[axis];
  const int stride = axis == 1 ? nx : nx * ny;
  const int base = axis == 1 ? x0 + nx * ny * other : x0 + nx * other;
  const bool xok = x0 < nx;  // nx is a multiple of VW
  const int start = w * CH;
  const int len = FULL ? CH : max(0, min(CH, nl - start));
  const T lam = a.co.lam;
  const T *pw = a.co.pw;
  const int o0 = base + start * stride;
  T v[CH][VW];
  // EARLY: the epilogue's old values (u^n or p) are loaded with the
  // right-hand sides, so their latency hides behind the solve
  constexpr bool EARLY = PRO == PRO_LOAD && EPI != EPI_STORE;
  T old[EARLY ? CH : 1][VW];
  if (PRO == PRO_LOAD) {
#pragma unroll
    for (int e = 0; e < CH; ++e) {
      if (xok && (FULL || e < len)) ldv<VW>(Fin + o0 + e * stride, v[e]);
      else {
#pragma unroll
        for (int c = 0; c < VW; ++c) v[e][c] = T(0);
      }
    }
    if (EARLY) {
      const T *tgt = EPI == EPI_ADDU ? a.uo[comp] : a.p;
#pragma unroll
      for (int e = 0; e < CH; ++e)
        if (xok && (FULL || e < len)) ldv<VW>(tgt + o0 + e * stride, old[EARLY ? e : 0]);
    }
  } else {
    // Step 3e right-hand side -rho/dt D.u^{n+1}, accumulated in v axis by
    // axis in the order of div_at (x, y, z) from loads alone, so that the
    // loads of a phase are all independent and none waits behind a store;
    // D.u^{n+1} itself is parked in shared memory for the update of p and D.u
    // after the solve (sweep_s_div_tail)
    const int nz = a.dim == 3 ? a.n[2] : 1;
    // x part: the face after a lane's last column is the next lane's first
    // column; the last lane of the CTA, and the lane that ends the row (which
    // wraps to column 0), load it
    {
      const int xe = x0 + VW == nx ? -x0 : VW;
      const bool xload = lane == 31 || x0 + VW == nx;
#pragma unroll
      for (int e = 0; e < CH; ++e) {
        const bool ok = xok && (FULL || e < len);
        const int o = o0 + e * stride;
        T u0[VW];
#pragma unroll
        for (int c = 0; c < VW; ++c) u0[c] = T(0);
        if (ok) ldv_ro<VW>(a.u[0] + o, u0);
        const T nb = __shfl_down_sync(IBG_FULL, u0[0], 1);
        const T ue = ok && xload ? ld_ro(a.u[0] + o + xe) : nb;
#pragma unroll
        for (int c = 0; c < VW; ++c) {
          const T up = c + 1 < VW ? u0[c + 1 < VW ? c + 1 : 0] : ue;
          v[e][c] = ok ? (up - u0[c]) * a.inv_h[0] : T(0);
        }
      }
    }
    // the component along the line (v on y lines, w on z lines): its
    // neighbour is the chunk's next element, after the chunk the next chunk's
    // first element (element 0 at the end of the line)
    auto along = [&](const T *f, T ih) {
      const bool any = xok && (FULL || len > 0);
      const int tn = start + len < nl ? start + len : 0;
      T cur[VW], nxt[VW];
#pragma unroll
      for (int c = 0; c < VW; ++c) cur[c] = nxt[c] = T(0);
      if (any) {
        ldv_ro<VW>(f + o0, cur);
        ldv_ro<VW>(f + base + tn * stride, nxt);
      }
#pragma unroll
      for (int e = 0; e < CH; ++e) {
        const bool ok = xok && (FULL || e < len);
        T nb[VW];
#pragma unroll
        for (int c = 0; c < VW; ++c) nb[c] = nxt[c];
        if (e + 1 < CH && (FULL || e + 1 < len) && xok) ldv_ro<VW>(f + o0 + (e + 1) * stride, nb);
        if (ok) {
#pragma unroll
          for (int c = 0; c < VW; ++c) v[e][c] += (nb[c] - cur[c]) * ih;
        }
#pragma unroll
        for (int c = 0; c < VW; ++c) cur[c] = nb[c];
      }
    };
    // a component across the lines: its neighbour lies `off` elements away
    // (the line's fixed coordinate + 1, periodic)
    auto across = [&](const T *f, int off, T ih) {
#pragma unroll
      for (int e = 0; e < CH; ++e)
        if (xok && (FULL || e < len)) {
          const int o = o0 + e * stride;
          T f0[VW], f1[VW];
          ldv_ro<VW>(f + o, f0);
          ldv_ro<VW>(f + o + off, f1);
#pragma unroll
          for (int c = 0; c < VW; ++c) v[e][c] += (f1[c] - f0[c]) * ih;
        }
    };
    if (axis == 1) along(a.u[1], a.inv_h[1]);
    else across(a.u[1], other + 1 == ny ? nx * (1 - ny) : nx, a.inv_h[1]);
    if (a.dim == 3) {
      if (axis == 2) along(a.u[2], a.inv_h[2]);
      else across(a.u[2], other + 1 == nz ? nx * ny * (1 - nz) : nx * ny, a.inv_h[2]);
    }
    T *sd = reinterpret_cast<T *>(ibg_sweep_dyn);
#pragma unroll
    for (int e = 0; e < CH; ++e)
#pragma unroll
      for (int c = 0; c < VW; ++c) {
        sd[(e * VW + c) * (32 * W) + threadIdx.x] = v[e][c];
        v[e][c] = a.pro_scale * v[e][c];
      }
  }
  __syncthreads();  // lp
  const T gCH = lp[CH];
  // forward factor (I - lam S) y = b: local pass, chunk scan, correction
  {
    T z[VW];
#pragma unroll
    for (int c = 0; c < VW; ++c) z[c] = T(0);
#pragma unroll
    for (int e = 0; e < CH; ++e)
      if (FULL || e < len) {
#pragma unroll
        for (int c = 0; c < VW; ++c) v[e][c] = z[c] = fma(lam, z[c], v[e][c]);
      }
#pragma unroll
    for (int c = 0; c < VW; ++c) sz[w][c][lane] = z[c];
  }
  __syncthreads();
  const T pstart = ld_ro(pw + min(start, nl));
  if (SCAN1) {
    if (w == 0) {
#pragma unroll
      for (int c = 0; c < VW; ++c) {
        T run = T(0);
        for (int q = 0; q < W; ++q) {
          const T zq = sz[q][c][lane];
          sz[q][c][lane] = run;
          run = fma(run, FULL ? gCH : ld_ro(pw + max(0, min(CH, nl - q * CH))), zq);
        }
        stot[c][lane] = run;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < VW; ++c) {
    T cin = T(0), tot;
    if (SCAN1) {
      cin = sz[w][c][lane];
      tot = stot[c][lane];
    } else {
      for (int q = 0; q < w; ++q)
        cin = fma(cin, FULL ? gCH : ld_ro(pw + max(0, min(CH, nl - q * CH))), sz[q][c][lane]);
      tot = cin;
      for (int q = w; q < W; ++q)
        tot = fma(tot, FULL ? gCH : ld_ro(pw + max(0, min(CH, nl - q * CH))), sz[q][c][lane]);
    }
    const T t = EXT ? wrap_term<true>(a.co, min(start, nl), tot, cin) : fma(pstart, tot * a.co.inv_1m, cin);
#pragma unroll
    for (int e = 0; e < CH; ++e)
      if (FULL || e < len) v[e][c] = fma(lp[e + 1], t, v[e][c]);
  }
  __syncthreads();
  // backward factor (I - lam S^{-1}) x = y
  {
    T z[VW];
#pragma unroll
    for (int c = 0; c < VW; ++c) z[c] = T(0);
#pragma unroll
    for (int e = CH - 1; e >= 0; --e)
      if (FULL || e < len) {
#pragma unroll
        for (int c = 0; c < VW; ++c) v[e][c] = z[c] = fma(lam, z[c], v[e][c]);
      }
#pragma unroll
    for (int c = 0; c < VW; ++c) sz[w][c][lane] = z[c];
  }
  __syncthreads();
  if (SCAN1) {
    if (w == 0) {
#pragma unroll
      for (int c = 0; c < VW; ++c) {
        T run = T(0);
        for (int q = W - 1; q >= 0; --q) {
          const T zq = sz[q][c][lane];
          sz[q][c][lane] = run;
          run = fma(run, FULL ? gCH : ld_ro(pw + max(0, min(CH, nl - q * CH))), zq);
        }
        stot[c][lane] = run;
      }
    }
    __syncthreads();
  }
  if (FULL || len > 0) {
    const T pend = ld_ro(pw + (nl - start - len));
#pragma unroll
    for (int c = 0; c < VW; ++c) {
      T cin = T(0), tot;
      if (SCAN1) {
        cin = sz[w][c][lane];
        tot = stot[c][lane];
      } else {
        for (int q = W - 1; q > w; --q)
          cin = fma(cin, FULL ? gCH : ld_ro(pw + max(0, min(CH, nl - q * CH))), sz[q][c][lane]);
        tot = cin;
        for (int q = w; q >= 0; --q)
          tot = fma(tot, FULL ? gCH : ld_ro(pw + max(0, min(CH, nl - q * CH))), sz[q][c][lane]);
      }
      const T t = EXT ? wrap_term<true>(a.co, nl - start - len, tot, cin) : fma(pend, tot * a.co.inv_1m, cin);
#pragma unroll
      for (int e = 0; e < CH; ++e)
        if (FULL || e < len) {
          const int pe = FULL ? CH - e : max(0, len - e);
          v[e][c] = fma(lp[pe], t, v[e][c]);
        }
    }
  }
  if (!xok) return;
  // the scale 1/c (EPI_ADDU folds it into the sum); skipped in the unscaled
  // sweeps of a chain
  const T sc = a.co.scale;
  if (EPI != EPI_ADDU && sc != T(1)) {
#pragma unroll
    for (int e = 0; e < CH; ++e)
#pragma unroll
      for (int c = 0; c < VW; ++c) v[e][c] *= sc;
  }
  if (EPI == EPI_STORE) {
#pragma unroll
    for (int e = 0; e < CH; ++e)
      if (FULL || e < len) stv<VW>(F + o0 + e * stride, v[e]);
    if (PRO == PRO_DIV) {
      // sweep_s_div_tail: Step 3f without psi, p <- p_keep p - chi mu / 2
      // (D.u^{n+1} + D.u^n), and D.u^n <- D.u^{n+1} (parked in shared memory
      // by the prologue), G elements per batch of loads
      const T *sd = reinterpret_cast<const T *>(ibg_sweep_dyn);
      constexpr int G = 16 / VW < CH ? 16 / VW : CH;
#pragma unroll
      for (int e0 = 0; e0 < CH; e0 += G) {
        T dv[G][VW], pv[G][VW];
#pragma unroll
        for (int g = 0; g < G; ++g)
          if (FULL || e0 + g < len) {
            ldv_ro<VW>(a.div + o0 + (e0 + g) * stride, dv[g]);
            ldv_ro<VW>(a.p + o0 + (e0 + g) * stride, pv[g]);
          }
#pragma unroll
        for (int g = 0; g < G; ++g)
          if (FULL || e0 + g < len) {
            T dn[VW], pn[VW];
#pragma unroll
            for (int c = 0; c < VW; ++c) {
              const T d = sd[((e0 + g) * VW + c) * (32 * W) + threadIdx.x];
              dn[c] = d;
              pn[c] = kept_p(a, pv[g][c]) - a.chi_mu_half * (d + dv[g][c]);
            }
            stv<VW>(a.div + o0 + (e0 + g) * stride, dn);
            stv<VW>(a.p + o0 + (e0 + g) * stride, pn);
          }
      }
    }
  } else {
    // psi stores first, then every load of the old values, then the sums:
    // no load waits behind a store
    T *tgt = EPI == EPI_ADDU ? a.uo[comp] : a.p;
    if (EPI == EPI_P) {
#pragma unroll
      for (int e = 0; e < CH; ++e)
        if (FULL || e < len) stv<VW>(F + o0 + e * stride, v[e]);
    }
#pragma unroll
    for (int e = 0; e < CH; ++e)
      if (FULL || e < len) {
        T ol[VW];
        if (EARLY) {
#pragma unroll
          for (int c = 0; c < VW; ++c) ol[c] = old[EARLY ? e : 0][c];
        } else {
          ldv<VW>(tgt + o0 + e * stride, ol);
        }
#pragma unroll
        for (int c = 0; c < VW; ++c) v[e][c] = EPI == EPI_ADDU ? fma(v[e][c], sc, ol[c]) : v[e][c] + ol[c];
      }
#pragma unroll
    for (int e = 0; e < CH; ++e)
      if (FULL || e < len) stv<VW>(tgt + o0 + e * stride, v[e]);
  }
}
template <typename T, int VW, int CH, int W, int PRO, int EPI, bool FULL, bool EXT>
__global__ void __launch_bounds__(32 * W) k_sweep_s(const SweepArgs<T> a, const int axis) {
  pdl_wait();
  pdl_release();
  sweep_s_body<T, VW, CH, W, PRO, EPI, FULL, EXT>(a, axis, hw_blk());
}
template <typename T, int VW, int CH, int W, int PRO, int EPI, bool FULL, bool EXT>
__global__ void __launch_bounds__(32 * W) k_sweep_s_b(const __grid_constant__ Batch<SweepArgs<T>> Bt,
                                                      const int axis) {
  pdl_wait();
  pdl_release();
  Blk b;
  const int i = batch_member(Bt, b);
  sweep_s_body<T, VW, CH, W, PRO, EPI, FULL, EXT>(Bt.a[i], axis, b);
}

// Sweep configurations.  Strided lines (axes 1, 2): VW adjacent x columns
// per thread, CH elements per warp chunk, W warps per line.  x lines: the
// grid is capped at XCAP[i] CTAs of 8 warps per SM (warps loop over lines).
struct StridedCfg {
  int vw, ch, w;
};
__host__ __device__ constexpr StridedCfg strided_cfg(int i) {
  return i == 0 ? StridedCfg{1, 8, 8}
       : i == 1 ? StridedCfg{2, 8, 8}
       : i == 2 ? StridedCfg{4, 8, 8}
       : i == 3 ? StridedCfg{1, 16, 8}
       : i == 4 ? StridedCfg{2, 8, 16}
       : i == 5 ? StridedCfg{4, 8, 16}
       : i == 6 ? StridedCfg{1, 16, 16}
       : i == 7 ? StridedCfg{2, 16, 16}
       : i == 8 ? StridedCfg{1, 16, 32}
       : i == 9 ? StridedCfg{2, 16, 32}
       : i == 10 ? StridedCfg{1, 32, 16}
       // (id 11 is the TMA kernel, kTmaCfg)
       : i == 12 ? StridedCfg{1, 32, 4}
       : i == 13 ? StridedCfg{2, 16, 8}
                 : StridedCfg{1, 32, 8};
}
constexpr int kStridedCfgs = 15;  // ids 0 .. 14 except kTmaCfg
constexpr int kXCaps = 4;
__host__ __device__ constexpr int xcap(int i) { return i == 0 ? 2 : i == 1 ? 4 : i == 2 ? 8 : 1 << 20; }

// Whether strided configuration i can run this sweep: it must cover the line
// with less than twice its length (n <= CH W < 2n; the smallest shape,
// CH = 8 and W = 8, covers every shorter line), n_x must be a multiple of VW,
// and VW CH is at most 32 values per thread (FP64: VW = 1 only).
inline bool strided_cfg_ok(int i, int nl, int nx, bool dbl) {
  if (i < 0 || i >= kStridedCfgs || i == kTmaCfg) return false;
  const StridedCfg c = strided_cfg(i);
  const bool smallest = c.ch == 8 && c.w == 8;
  if (c.ch * c.w < nl || (!smallest && c.ch * c.w >= 2 * nl) || nx % c.vw) return false;
  if (dbl) return c.vw == 1 && i <= 10;  // the FP64 kernels are instantiated for ids 0, 3, 6, 8, 10
  return c.vw * c.ch <= 32;
}

// dynamic shared memory of a strided sweep with the divergence prologue: one
// value per element of the CTA's lines
inline size_t sweep_s_div_smem(int cfg, size_t elem) {
  const StridedCfg c = strided_cfg(cfg);
  return (size_t)c.ch * c.vw * 32 * c.w * elem;
}

// The default choice (no autotuning): the first valid configuration in the
// order of preference below.
inline int strided_cfg_default(int nl, int nx, bool dbl) {
  static const int pref_f[] = {3, 0, 6, 1, 4, 7, 9, 2, 5, 8, 10};
  static const int pref_d[] = {0, 3, 6, 10, 8};
  const int *pref = dbl ? pref_d : pref_f;
  const int np = dbl ? 5 : 11;
  for (int k = 0; k < np; ++k)
    if (strided_cfg_ok(pref[k], nl, nx, dbl)) return pref[k];
  return -1;
}

// line lengths 8 <= n <= 512 (checked by the caller); cfg < 0: default
template <typename T, int PRO, int EPI, bool EXT>
cudaError_t launch_sweep_t(int axis, int nfields, const SweepArgs<T> &a, cudaStream_t s, int cfg) {
  const int nl = a.n[axis];
  if (axis == 0) {
    const long long nlines = (long long)a.n[1] * (a.dim == 3 ? a.n[2] : 1);
    const long long ctas = (nlines + 7) / 8;
    const long long sms = device_sms(), cap = (sms > 0 ? sms : 152) * xcap(cfg < 0 || cfg >= kXCaps ? 1 : cfg);
    dim3 grid((unsigned)(ctas < cap ? ctas : cap), nfields);  // warps loop over lines
    const dim3 b(256);
    if (nl == 128) return launch_pdl(k_sweep_x<T, 1, PRO, EPI, true, EXT>, grid, b, 0, s, a);
    if (nl < 128) return launch_pdl(k_sweep_x<T, 1, PRO, EPI, false, EXT>, grid, b, 0, s, a);
    if (nl == 256) return launch_pdl(k_sweep_x<T, 2, PRO, EPI, true, EXT>, grid, b, 0, s, a);
    if (nl < 256) return launch_pdl(k_sweep_x<T, 2, PRO, EPI, false, EXT>, grid, b, 0, s, a);
    if (nl == 512) return launch_pdl(k_sweep_x<T, 4, PRO, EPI, true, EXT>, grid, b, 0, s, a);
    return launch_pdl(k_sweep_x<T, 4, PRO, EPI, false, EXT>, grid, b, 0, s, a);
  } else {
    const int other = axis == 1 ? (a.dim == 3 ? a.n[2] : 1) : a.n[1];
    const int nx = a.n[0];
    const bool dbl = sizeof(T) == 8;
    if (cfg < 0 || cfg >= kStridedCfgs || !strided_cfg_ok(cfg, nl, nx, dbl)) cfg = strided_cfg_default(nl, nx, dbl);
    auto grid = [&](int v) { return dim3((unsigned)((nx / v + 31) / 32), other, nfields); };
    const size_t smem = PRO == PRO_DIV ? sweep_s_div_smem(cfg, sizeof(T)) : 0;
    auto run = [&](auto kernel, int vw, int w) -> cudaError_t {
      if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
      }
      return launch_pdl(kernel, grid(vw), dim3(32 * w), smem, s, a, axis);
    };
#define IBG_S(I)                                                                 \
  case I: {                                                                      \
    constexpr StridedCfg c = strided_cfg(I);                                     \
    if (nl == c.ch * c.w) return run(k_sweep_s<T, c.vw, c.ch, c.w, PRO, EPI, true, EXT>, c.vw, c.w); \
    return run(k_sweep_s<T, c.vw, c.ch, c.w, PRO, EPI, false, EXT>, c.vw, c.w);  \
  }
    if constexpr (sizeof(T) == 8) {
      switch (cfg) { IBG_S(0) IBG_S(3) IBG_S(6) IBG_S(8) IBG_S(10) default: return cudaErrorInvalidValue; }
    } else {
      switch (cfg) {
        IBG_S(0) IBG_S(1) IBG_S(2) IBG_S(3) IBG_S(4) IBG_S(5) IBG_S(6) IBG_S(7) IBG_S(8) IBG_S(9) IBG_S(10)
        IBG_S(12) IBG_S(13) IBG_S(14)
        default: return cudaErrorInvalidValue;
      }
    }
#undef IBG_S
  }
  return cudaGetLastError();
}

// The same sweeps for n grids of one size class in batched launches (the
// register kernels only; every member has the same n, precision and dim)
template <typename T, int PRO, int EPI, bool EXT>
cudaError_t launch_sweep_batch_t(int axis, int nfields, const SweepArgs<T> *a, int n, cudaStream_t s, int cfg) {
  const SweepArgs<T> &a0 = a[0];
  const int nl = a0.n[axis];
  std::vector<dim3> g(n);
  if (axis == 0) {
    const long long nlines = (long long)a0.n[1] * (a0.dim == 3 ? a0.n[2] : 1);
    const long long ctas = (nlines + 7) / 8;
    const long long sms = device_sms(), cap = (sms > 0 ? sms : 152) * xcap(cfg < 0 || cfg >= kXCaps ? 1 : cfg);
    for (int i = 0; i < n; ++i) g[i] = dim3((unsigned)(ctas < cap ? ctas : cap), nfields);
    const dim3 b(256);
    if (nl == 128) return launch_batch(k_sweep_x_b<T, 1, PRO, EPI, true, EXT>, a, g.data(), n, b, s);
    if (nl < 128) return launch_batch(k_sweep_x_b<T, 1, PRO, EPI, false, EXT>, a, g.data(), n, b, s);
    if (nl == 256) return launch_batch(k_sweep_x_b<T, 2, PRO, EPI, true, EXT>, a, g.data(), n, b, s);
    if (nl < 256) return launch_batch(k_sweep_x_b<T, 2, PRO, EPI, false, EXT>, a, g.data(), n, b, s);
    if (nl == 512) return launch_batch(k_sweep_x_b<T, 4, PRO, EPI, true, EXT>, a, g.data(), n, b, s);
    return launch_batch(k_sweep_x_b<T, 4, PRO, EPI, false, EXT>, a, g.data(), n, b, s);
  }
  const int other = axis == 1 ? (a0.dim == 3 ? a0.n[2] : 1) : a0.n[1];
  const int nx = a0.n[0];
  const bool dbl = sizeof(T) == 8;
  if (cfg < 0 || cfg >= kStridedCfgs || !strided_cfg_ok(cfg, nl, nx, dbl)) cfg = strided_cfg_default(nl, nx, dbl);
  auto grids = [&](int v) {
    for (int i = 0; i < n; ++i) g[i] = dim3((unsigned)((nx / v + 31) / 32), other, nfields);
    return g.data();
  };
  const size_t smem = PRO == PRO_DIV ? sweep_s_div_smem(cfg, sizeof(T)) : 0;
  auto run = [&](auto kernel, int vw, int w) -> cudaError_t {
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    return launch_batch_smem(kernel, a, grids(vw), n, dim3(32 * w), smem, s, axis);
  };
#define IBG_SB(I)                                                                  \
  case I: {                                                                        \
    constexpr StridedCfg c = strided_cfg(I);                                       \
    if (nl == c.ch * c.w) return run(k_sweep_s_b<T, c.vw, c.ch, c.w, PRO, EPI, true, EXT>, c.vw, c.w); \
    return run(k_sweep_s_b<T, c.vw, c.ch, c.w, PRO, EPI, false, EXT>, c.vw, c.w);  \
  }
  if constexpr (sizeof(T) == 8) {
    switch (cfg) { IBG_SB(0) IBG_SB(3) IBG_SB(6) IBG_SB(8) IBG_SB(10) default: return cudaErrorInvalidValue; }
  } else {
    switch (cfg) {
      IBG_SB(0) IBG_SB(1) IBG_SB(2) IBG_SB(3) IBG_SB(4) IBG_SB(5) IBG_SB(6) IBG_SB(7) IBG_SB(8) IBG_SB(9) IBG_SB(10)
      IBG_SB(12) IBG_SB(13) IBG_SB(14)
      default: return cudaErrorInvalidValue;
    }
  }
#undef IBG_SB
}

template <typename T, bool EXT>
cudaError_t launch_sweep_batch_impl(int axis, int pro, int epi, int nfields, const SweepArgs<T> *a, int n,
                                    cudaStream_t s, int cfg) {
  if (n < 1) return cudaSuccess;
  if (pro == PRO_LOAD && epi == EPI_STORE) return launch_sweep_batch_t<T, PRO_LOAD, EPI_STORE, EXT>(axis, nfields, a, n, s, cfg);
  if (pro == PRO_LOAD && epi == EPI_ADDU) return launch_sweep_batch_t<T, PRO_LOAD, EPI_ADDU, EXT>(axis, nfields, a, n, s, cfg);
  if (pro == PRO_DIV && epi == EPI_STORE) return launch_sweep_batch_t<T, PRO_DIV, EPI_STORE, EXT>(axis, nfields, a, n, s, cfg);
  if (pro == PRO_LOAD && epi == EPI_P) return launch_sweep_batch_t<T, PRO_LOAD, EPI_P, EXT>(axis, nfields, a, n, s, cfg);
  return cudaErrorInvalidValue;
}

template <typename T, bool EXT>
cudaError_t launch_sweep_impl(int axis, int pro, int epi, int nfields, const SweepArgs<T> &a, cudaStream_t s,
                              int cfg) {
  if (pro == PRO_LOAD && epi == EPI_STORE) return launch_sweep_t<T, PRO_LOAD, EPI_STORE, EXT>(axis, nfields, a, s, cfg);
  if (pro == PRO_LOAD && epi == EPI_ADDU) return launch_sweep_t<T, PRO_LOAD, EPI_ADDU, EXT>(axis, nfields, a, s, cfg);
  if (pro == PRO_DIV && epi == EPI_STORE) return launch_sweep_t<T, PRO_DIV, EPI_STORE, EXT>(axis, nfields, a, s, cfg);
  if (pro == PRO_LOAD && epi == EPI_P) return launch_sweep_t<T, PRO_LOAD, EPI_P, EXT>(axis, nfields, a, s, cfg);
  return cudaErrorInvalidValue;
}

}  // namespace ibg
