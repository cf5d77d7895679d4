// Marker kernels of one IB-GM step for sm_103a: interpolation (Step 1a), the
// AB2 marker update and half position (Steps 1b-1c), the force connections
// (Step 2a) and spreading (Step 2b).
//
// Positions are FP64.  Everything that needs FP64 arithmetic on positions
// (the AB2 update and locating a marker on the grid) runs with one thread per
// marker, where every lane does useful work: on GB300 a warp instruction on
// the FP64 pipe costs the same whether 1 or 32 lanes are active.  The stencil
// kernels (interpolation, spreading) then work in the field precision only,
// from a stored location: for every axis a and MAC offset o (0 on the
// component's own axis, 1/2 on the others) the index of the first of the 4
// stencil nodes and their 4 weights.
#include <math.h>

#include <vector>

#include "ib_internal.cuh"

namespace ibg {

__device__ __forceinline__ float cospi_t(float x) { return cospif(x); }
__device__ __forceinline__ double cospi_t(double x) { return cospi(x); }

// i + d for a node index i in [0, n) and a stencil step 0 <= d <= 3 < n,
// periodic: one compare and subtract (the stored first nodes are wrapped)
__device__ __forceinline__ int step_wrap(int i, int n) { return i >= n ? i - n : i; }
// i mod n in [0, n) for any i (the first stencil node of an unwrapped position)
__device__ __forceinline__ int mod_n(int i, int n) {
  if (i >= 0 && i < n) return i;
  const int r = i % n;
  return r < 0 ? r + n : r;
}

// Locations of one coordinate for both MAC offsets from a single FP64
// product: x = X/h, i0 = floor(x), f0 = x - i0; for the half-cell offset the
// fraction is f0 - 1/2 (same cell) or f0 + 1/2 (previous cell).
template <typename T>
__device__ __forceinline__ void locate2(double X, double inv_h, int &b0, T &f0, int &b1, T &f1) {
  const double x = X * inv_h;
  const double fl = floor(x);
  f0 = (T)(x - fl);
  b0 = (int)fl - 1;
  if (f0 >= T(0.5)) {
    f1 = f0 - T(0.5);
    b1 = b0;
  } else {
    f1 = f0 + T(0.5);
    b1 = b0 - 1;
  }
}

// Weights of the 4 stencil nodes, at r = -1-f, -f, 1-f, 2-f.  Both branches
// of the 4-point kernel of eq. (discretedelta) share q = sqrt(1 + 4f - 4f^2)
// on these nodes: (3-2f-q)/8, (3-2f+q)/8, (1+2f+q)/8, (1+2f-q)/8 (sum 1).
// The cosine kernel is (1 + cos(pi r / 2)) / 4.
template <typename T>
__device__ __forceinline__ void weights(T f, int kernel, T (&w)[4]) {
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
}

// Location of coordinate X on axis a for both MAC offsets: first stencil
// node b[2a + o], wrapped into [0, n_a) (positions are kept unwrapped; the
// force kernel's nearest-image shift is exact for any whole-period offset),
// and the 4 weights w[2a + o][0..3] (stored as 4 consecutive values of the
// field precision).
// With lf, the own-axis fraction f0 is stored as well.
template <typename T>
__device__ __forceinline__ void store_location(const MarkerArgs &m, double X, int a, long long k, int32_t *lb,
                                               T *lw, T *lf = nullptr) {
  int b0, b1;
  T f0, f1, w[4];
  locate2<T>(X, m.inv_h[a], b0, f0, b1, f1);
  const long long s0 = (2 * a) * m.nm + k, s1 = (2 * a + 1) * m.nm + k;
  lb[s0] = mod_n(b0, m.n[a]);
  lb[s1] = mod_n(b1, m.n[a]);
  if (lf) lf[a * m.nm + k] = f0;
  weights<T>(f0, m.kernel, w);
  st4(lw + 4 * s0, w);
  weights<T>(f1, m.kernel, w);
  st4(lw + 4 * s1, w);
}

// Locations of every marker at its positions Xs (one thread per marker).
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_locate(const MarkerArgs m, double *const X0, double *const X1,
                                                double *const X2, int32_t *lb, T *lw) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m.nm) return;
  const double *Xs[3] = {X0, X1, X2};
#pragma unroll
  for (int a = 0; a < DIM; ++a) store_location<T>(m, Xs[a][k], a, k, lb, lw);
}

// Steps 1b-1c after interpolation, one thread per marker:
//   V = 3/2 U^n - 1/2 U^{n-1} (U^0 at n = 0), X^{n+1} = X^n + dt V,
//   X^{n+1/2} = (X^{n+1} + X^n) / 2, U^{n-1} <- U^n,
// and the grid locations of X^{n+1/2} (spreading, this step) and of X^{n+1}
// (interpolation, next step).
template <typename T, int DIM>
__device__ __forceinline__ void update_body(const MarkerArgs &m, const Blk &B) {
  const unsigned t = B.x * blockDim.x + threadIdx.x;
  const unsigned k = t / DIM;
  const int c = (int)(t - k * DIM);
  if (k >= (unsigned)m.nm) return;
  const unsigned nm = (unsigned)m.nm;
  const T Ut = ((const T *)m.U[c])[k];
  const double U = (double)Ut;
  const double vel = m.first ? U : 1.5 * U - 0.5 * (double)((const T *)m.Uold[c])[k];
  const double Xc = m.X[c][k];
  const double Xn = Xc + m.dt * vel;
  const double Xh = 0.5 * (Xn + Xc);
  m.Xh[c][k] = Xh;
  m.X[c][k] = Xn;
  ((T *)m.Uold[c])[k] = Ut;
  (void)nm;
  store_location<T>(m, Xh, c, k, m.locS_b, (T *)m.locS_w, (T *)m.locS_f);
  store_location<T>(m, Xn, c, k, m.locI_b, (T *)m.locI_w);
}
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_update(const MarkerArgs m) {
  pdl_wait();
  pdl_release();
  update_body<T, DIM>(m, hw_blk());
}
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_update_b(const __grid_constant__ Batch<MarkerArgs> Bt) {
  pdl_wait();
  pdl_release();
  Blk b;
  const int i = batch_member(Bt, b);
  update_body<T, DIM>(Bt.a[i], b);
}

// Lane groups for the 4^d-node stencils: one group of ROWS lanes per
// (marker, component c) (16 in 3D, 4 in 2D); lane r owns the stencil row
// (y, z) = (r & 3, r >> 2) and its 4 nodes along x.  Every lane reads the
// stored locations and weights it needs.
template <typename T, int DIM>
struct StencilLanes {
  static constexpr int ROWS = DIM == 3 ? 16 : 4;
  unsigned k;  // marker
  int c, row, jy, kz;
  bool valid;
  T wx[4], wrow;  // x weights; product of this row's y (and z) weights
  int bx, yrow, zrow;
  // pair: the (marker, component) index k d + c; row: this lane's stencil row
  __device__ __forceinline__ StencilLanes(const MarkerArgs &m, const int32_t *lb, const T *lw, unsigned pair,
                                          int row_) {
    row = row_;
    k = pair / DIM;
    c = (int)(pair - k * DIM);
    valid = k < (unsigned)m.nm;
    jy = row & 3;
    kz = DIM == 3 ? row >> 2 : 0;
    bx = yrow = zrow = 0;
    wrow = T(0);
    if (!valid) return;
    const unsigned nm = (unsigned)m.nm;
    unsigned s = 2 * 0 + (c == 0 ? 0 : 1);
    bx = lb[s * nm + k];
    ld4(lw + 4 * (s * nm + k), wx);
    s = 2 * 1 + (c == 1 ? 0 : 1);
    yrow = step_wrap(lb[s * nm + k] + jy, m.n[1]);
    wrow = lw[4 * (s * nm + k) + jy];
    if (DIM == 3) {
      s = 2 * 2 + (c == 2 ? 0 : 1);
      zrow = step_wrap(lb[s * nm + k] + kz, m.n[2]);
      wrow *= lw[4 * (s * nm + k) + kz];
    }
  }
  __device__ __forceinline__ long long row_offset(const MarkerArgs &m) const {
    return ((long long)zrow * m.n[1] + yrow) * m.n[0];
  }
};

// 3D spreading stencils, one warp per (marker, component c): lane l owns the node
// q = l & 3 along x of the stencil rows r = l >> 2 and r + 8, (y, z) =
// (r & 3, r >> 2), so one warp instruction touches 4 consecutive nodes of 8
// rows (a few cache sectors) instead of 16 lanes' scattered 128-bit windows.
// w0, w1 are the products of the node's three 1-D weights.
template <typename T>
struct StencilNodes3 {
  unsigned k;
  int c;
  bool valid;
  T w0, w1;
  unsigned o0, o1;  // element offsets of the two nodes (fields hold < 2^31 elements)
  StencilNodes3() = default;
  // gw: the (marker, component) index k 3 + c
  __device__ __forceinline__ StencilNodes3(const MarkerArgs &m, const int32_t *lb, const T *lw, unsigned gw) {
    const int lane = threadIdx.x & 31;
    k = gw / 3;
    c = (int)(gw - k * 3);
    valid = k < (unsigned)m.nm;
    w0 = w1 = T(0);
    o0 = o1 = 0;
    if (!valid) return;
    const unsigned nm = (unsigned)m.nm;
    const int q = lane & 3, jy = (lane >> 2) & 3, kz = lane >> 4;
    const unsigned sx = c == 0 ? 0 : 1, sy = c == 1 ? 2 : 3, sz = c == 2 ? 4 : 5;
    const int x = step_wrap(lb[sx * nm + k] + q, m.n[0]);
    const int y = step_wrap(lb[sy * nm + k] + jy, m.n[1]);
    const int bz = lb[sz * nm + k];
    const int z0 = step_wrap(bz + kz, m.n[2]), z1 = step_wrap(bz + kz + 2, m.n[2]);
    const T wxy = lw[4 * (sx * nm + k) + q] * lw[4 * (sy * nm + k) + jy];
    w0 = wxy * lw[4 * (sz * nm + k) + kz];
    w1 = wxy * lw[4 * (sz * nm + k) + kz + 2];
    o0 = ((unsigned)z0 * m.n[1] + y) * m.n[0] + x;
    o1 = ((unsigned)z1 * m.n[1] + y) * m.n[0] + x;
  }
};

// 4 consecutive values r[xs .. xs+3] of a row, periodic in x: one aligned
// 256-bit load when the window lies in one 8-float block (5 of 8 offsets,
// n_x divisible by 8), else aligned 128-bit loads (the second only when xs is
// not 4-aligned) when the 8-float block around xs lies inside the row
__device__ __forceinline__ void row4(const float *r, int xs, int nx, float (&v)[4]) {
  const int a8 = xs & ~7, off8 = xs - a8;
  if ((nx & 7) == 0 && off8 <= 4) {
    float t[8];
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(t[0]), "=f"(t[1]), "=f"(t[2]), "=f"(t[3]), "=f"(t[4]), "=f"(t[5]), "=f"(t[6]), "=f"(t[7])
                 : "l"(r + a8));
#pragma unroll
    for (int i = 0; i < 4; ++i)
      v[i] = off8 == 0 ? t[i] : off8 == 1 ? t[i + 1] : off8 == 2 ? t[i + 2] : off8 == 3 ? t[i + 3] : t[i + 4];
    return;
  }
  const int a0 = xs & ~3;
  if ((nx & 3) == 0 && a0 + 8 <= nx) {
    const int off = xs - a0;
    const float4 p = __ldg(reinterpret_cast<const float4 *>(r + a0));
    const float4 q = off ? __ldg(reinterpret_cast<const float4 *>(r + a0 + 4)) : p;
    const float t[8] = {p.x, p.y, p.z, p.w, q.x, q.y, q.z, q.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = off == 0 ? t[i] : off == 1 ? t[i + 1] : off == 2 ? t[i + 2] : t[i + 3];
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __ldg(r + (xs + i < nx ? xs + i : xs + i - nx));
  }
}
__device__ __forceinline__ void row4(const double *r, int xs, int nx, double (&v)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __ldg(r + (xs + i < nx ? xs + i : xs + i - nx));
}

// r[xs .. xs+3] += v, periodic in x; 128-bit vector atomics when the 8-float
// block around xs lies inside the row (block lanes outside [xs, xs+3] add 0)
__device__ __forceinline__ void row4_add(float *r, int xs, int nx, const float (&v)[4]) {
  const int a0 = xs & ~3;
  if ((nx & 3) == 0 && a0 + 8 <= nx) {
    const int off = xs - a0;
    float t[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int q = i - off;
      t[i] = q == 0 ? v[0] : q == 1 ? v[1] : q == 2 ? v[2] : q == 3 ? v[3] : 0.0f;
    }
    atomicAdd(reinterpret_cast<float4 *>(r + a0), make_float4(t[0], t[1], t[2], t[3]));
    if (off) atomicAdd(reinterpret_cast<float4 *>(r + a0 + 4), make_float4(t[4], t[5], t[6], t[7]));
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) atomicAdd(r + (xs + i < nx ? xs + i : xs + i - nx), v[i]);
  }
}
__device__ __forceinline__ void row4_add(double *r, int xs, int nx, const double (&v)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) atomicAdd(r + (xs + i < nx ? xs + i : xs + i - nx), v[i]);
}

// (marker, component) pairs per lane group of k_interp and per warp of
// k_spread3: their loads are issued together, so that a group waits for one
// round of load latency per kInterpItems / kSpreadItems pairs.  Measured on
// GB300 (1 / 2 / 4 pairs): spreading 26.6 / 24.6 / 24.6 us at 128^3 and
// 287 / 251 / 236 us at 512^3 (8 x 64 002 markers); interpolation 20.7 / 21.1 /
// 23.0 us at 128^3 and 185 / 181 / 178 us at 512^3, so it keeps one pair at
// the size where it is on the step's critical path.
constexpr int kInterpItems = 1;
constexpr int kSpreadItems = 4;

// Step 1a: U_c = sum over the 4^d nodes of u_c(node) prod_a phi_a, at X^n.
template <typename T, int DIM>
__device__ __forceinline__ void interp_body(const MarkerArgs &m, const T *const u0, const T *const u1,
                                            const T *const u2, const Blk &B) {
  constexpr int ROWS = StencilLanes<T, DIM>::ROWS;
  // 32-bit index arithmetic: marker count * d * ROWS < 2^31 (checked on the host)
  const unsigned gt = B.x * blockDim.x + threadIdx.x;
  const unsigned grp = gt / ROWS;
  const int row = (int)(gt & (ROWS - 1));
  T s[kInterpItems];
  bool ok[kInterpItems];
  unsigned kk[kInterpItems];
  int cc[kInterpItems];
#pragma unroll
  for (int i = 0; i < kInterpItems; ++i) {
    StencilLanes<T, DIM> L(m, m.locI_b, (const T *)m.locI_w, grp * kInterpItems + i, row);
    ok[i] = L.valid;
    kk[i] = L.k;
    cc[i] = L.c;
    s[i] = T(0);
    if (L.valid) {
      const T *uc = L.c == 0 ? u0 : (L.c == 1 ? u1 : u2);
      T v[4];
      row4(uc + L.row_offset(m), L.bx, m.n[0], v);
      s[i] = (v[0] * L.wx[0] + v[1] * L.wx[1] + v[2] * L.wx[2] + v[3] * L.wx[3]) * L.wrow;
    }
  }
#pragma unroll
  for (int i = 0; i < kInterpItems; ++i) {
#pragma unroll
    for (int off = ROWS / 2; off > 0; off >>= 1) s[i] += __shfl_xor_sync(0xffffffffu, s[i], off);
    if (ok[i] && row == 0) ((T *)m.U[cc[i]])[kk[i]] = s[i];
  }
}
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_interp(const MarkerArgs m, const T *const u0, const T *const u1,
                                                const T *const u2) {
  pdl_wait();
  pdl_release();
  interp_body<T, DIM>(m, u0, u1, u2, hw_blk());
}
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_interp_b(const __grid_constant__ Batch<MarkerFieldArgs> Bt) {
  pdl_wait();
  pdl_release();
  Blk b;
  const MarkerFieldArgs &A = Bt.a[batch_member(Bt, b)];
  interp_body<T, DIM>(A.m, (const T *)A.f[0], (const T *)A.f[1], (const T *)A.f[2], b);
}

// Step 2a over the force connections at X^{n+1/2}: 8 lanes per marker share
// its CSR row (lane j takes connections j, j+8, ...) and add their partial
// forces with shuffles; the spring arithmetic runs in the field precision.
// The difference X_b - X_a, reduced to the nearest periodic image, comes
//   FRAC = false: from the FP64 positions;
//   FRAC = true (FP32 fields): from the stored locations of X^{n+1/2},
//     X_q = h_q (i_q + 1 + f_q) with the integer first stencil node i_q and
//     the fraction f_q in [0, 1): X_b - X_a = h_q (di + df) with the integer
//     di = i_b - i_a, shifted by whole periods n_q in integer arithmetic, and
//     the FP32 fraction difference df.  No FP64 instruction, and the same
//     accuracy as rounding the FP64 difference to FP32.
template <typename T, int DIM, bool FRAC>
__device__ __forceinline__ void force_body(const MarkerArgs &m, const Blk &B) {
  const unsigned gt = B.x * blockDim.x + threadIdx.x;
  const unsigned a = gt >> 3;
  const int lane8 = (int)(gt & 7);
  const bool valid = a < (unsigned)m.nm;
  T g[DIM];
#pragma unroll
  for (int q = 0; q < DIM; ++q) g[q] = T(0);
  if (valid) {
    const unsigned nm = (unsigned)m.nm;
    double xa[DIM];
    int ia[DIM];
    T fa[DIM];
#pragma unroll
    for (int q = 0; q < DIM; ++q) {
      if (FRAC) {
        ia[q] = m.locS_b[(2 * q) * nm + a];
        fa[q] = ((const T *)m.locS_f)[q * nm + a];
      } else {
        xa[q] = m.Xh[q][a];
      }
    }
    const T H = (T)m.H, invH = (T)(1.0 / m.H);
    const long long e1 = m.row[a + 1];
    for (long long e = m.row[a] + lane8; e < e1; e += 8) {
      const int b = m.col[e];
      T d[DIM], len2 = T(0);
#pragma unroll
      for (int q = 0; q < DIM; ++q) {
        if (FRAC) {
          const int di = m.locS_b[(2 * q) * nm + b] - ia[q];
          const T df = ((const T *)m.locS_f)[q * nm + b] - fa[q];
          const int sh = __float2int_rn(((float)di + (float)df) * m.inv_n32[q]);
          d[q] = ((T)(di - sh * m.n[q]) + df) * (T)m.h32[q];
        } else {
          d[q] = (T)(m.Xh[q][b] - xa[q]);
          d[q] -= H * rint(d[q] * invH);  // nearest periodic image
        }
        len2 += d[q] * d[q];
      }
      T scale, L;
      if (FRAC) {
        scale = ((const T *)m.kapT)[e];
        L = ((const T *)m.restT)[e];
      } else {
        scale = (T)m.kap[e];
        L = (T)m.rest[e];
      }
      if (L != T(0)) scale *= T(1) - L / sqrt(len2);
#pragma unroll
      for (int q = 0; q < DIM; ++q) g[q] += scale * d[q];
    }
  }
#pragma unroll
  for (int q = 0; q < DIM; ++q)
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) g[q] += __shfl_xor_sync(0xffffffffu, g[q], off);
  if (valid && lane8 < DIM) {
    const T gv = lane8 == 0 ? g[0] : (lane8 == 1 ? g[1] : g[DIM - 1]);
    ((T *)m.G[lane8])[a] = gv;
  }
}
template <typename T, int DIM, bool FRAC>
__global__ void __launch_bounds__(256) k_force(const MarkerArgs m) {
  pdl_wait();
  pdl_release();
  force_body<T, DIM, FRAC>(m, hw_blk());
}
template <typename T, int DIM, bool FRAC>
__global__ void __launch_bounds__(256) k_force_b(const __grid_constant__ Batch<MarkerArgs> Bt) {
  pdl_wait();
  pdl_release();
  Blk b;
  const int i = batch_member(Bt, b);
  force_body<T, DIM, FRAC>(Bt.a[i], b);
}

// Step 2b: f_c(node) += G_c prod_a phi_a / h^d at X^{n+1/2}, added as
// dt/rho f_c into the momentum increment R that the right-hand-side kernel
// stored (Step 3b), with global atomics.  This form (used in 2D) gives each
// (marker, c) a lane group, one row per lane, 128-bit vector atomics per row
// where the row segment allows; 3D uses k_spread3 below.  Markers are
// numbered in Morton order of their initial positions, so neighbouring groups
// update neighbouring nodes.
template <typename T, int DIM>
__device__ __forceinline__ void spread_body(const MarkerArgs &m, T *const f0, T *const f1, T *const f2,
                                            const Blk &B) {
  constexpr int ROWS = StencilLanes<T, DIM>::ROWS;
  const unsigned gt = B.x * blockDim.x + threadIdx.x;
  StencilLanes<T, DIM> L(m, m.locS_b, (const T *)m.locS_w, gt / ROWS, (int)(gt & (ROWS - 1)));
  if (!L.valid) return;
  T *fc = L.c == 0 ? f0 : (L.c == 1 ? f1 : f2);
  const T val = ((const T *)m.G[L.c])[L.k] * (T)m.spread_scale * L.wrow;
  T v[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = val * L.wx[i];
  row4_add(fc + L.row_offset(m), L.bx, m.n[0], v);
}
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_spread(const MarkerArgs m, T *const f0, T *const f1, T *const f2) {
  pdl_wait();
  pdl_release();
  spread_body<T, DIM>(m, f0, f1, f2, hw_blk());
}
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_spread_b(const __grid_constant__ Batch<MarkerFieldArgs> Bt) {
  pdl_wait();
  pdl_release();
  Blk b;
  const MarkerFieldArgs &A = Bt.a[batch_member(Bt, b)];
  spread_body<T, DIM>(A.m, (T *)A.f[0], (T *)A.f[1], (T *)A.f[2], b);
}

// The same spreading in 3D with a warp per (marker, c) and one scalar atomic
// per node: a warp's atomics then fall on a few sectors of 8 rows, which the
// L2 takes in fewer operations than 16 lanes' 128-bit vector atomics on
// scattered rows (26.6 against 28.5 us at 128^3).  Interpolation keeps the
// 16-lane groups: with a warp per (marker, c) it took 27.0 instead of 22.8 us.
template <typename T>
__device__ __forceinline__ void spread3_body(const MarkerArgs &m, T *const f0, T *const f1, T *const f2,
                                             const Blk &B) {
  // 32-bit unsigned warp index: at most 2^25 markers (checked on the host)
  const unsigned gw = (B.x * blockDim.x + threadIdx.x) >> 5;
  T gv[kSpreadItems];
  StencilNodes3<T> L[kSpreadItems];
#pragma unroll
  for (int i = 0; i < kSpreadItems; ++i) {
    L[i] = StencilNodes3<T>(m, m.locS_b, (const T *)m.locS_w, gw * kSpreadItems + i);
    gv[i] = L[i].valid ? ((const T *)m.G[L[i].c])[L[i].k] * (T)m.spread_scale : T(0);
  }
#pragma unroll
  for (int i = 0; i < kSpreadItems; ++i)
    if (L[i].valid) {
      T *fc = L[i].c == 0 ? f0 : (L[i].c == 1 ? f1 : f2);
      atomicAdd(fc + L[i].o0, gv[i] * L[i].w0);
      atomicAdd(fc + L[i].o1, gv[i] * L[i].w1);
    }
}
template <typename T>
__global__ void __launch_bounds__(256) k_spread3(const MarkerArgs m, T *const f0, T *const f1, T *const f2) {
  pdl_wait();
  pdl_release();
  spread3_body<T>(m, f0, f1, f2, hw_blk());
}
template <typename T>
__global__ void __launch_bounds__(256) k_spread3_b(const __grid_constant__ Batch<MarkerFieldArgs> Bt) {
  pdl_wait();
  pdl_release();
  Blk b;
  const MarkerFieldArgs &A = Bt.a[batch_member(Bt, b)];
  spread3_body<T>(A.m, (T *)A.f[0], (T *)A.f[1], (T *)A.f[2], b);
}

// marker positions between the caller's [n][dim] layout and the SoA arrays
// (internal marker k is the caller's marker perm[k])
__global__ void __launch_bounds__(256) k_markers_layout(double *aos, double *X0, double *X1, double *X2,
                                                        const int32_t *perm, long long nm, int dim, int to_soa) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nm * dim) return;
  const long long k = t / dim;
  const int c = (int)(t % dim);
  double *X = c == 0 ? X0 : (c == 1 ? X1 : X2);
  const long long o = (long long)perm[k] * dim + c;
  if (to_soa) X[k] = aos[o];
  else aos[o] = X[k];
}

// ---------------------------------------------------------------------------
// launchers

static inline unsigned nblocks(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : b);
}

// CTA size of the update and force kernels: at 128^3 they run below one wave
// (41 k markers), and 128-thread CTAs spread their work evenly over the SMs
constexpr int kMarkerCta = 128;

template <typename T>
cudaError_t launch_locate(const MarkerArgs &m, cudaStream_t s) {
  if (m.nm == 0) return cudaSuccess;
  if (m.dim == 2) k_locate<T, 2><<<nblocks(m.nm, 256), 256, 0, s>>>(m, m.X[0], m.X[1], m.X[1], m.locI_b, (T *)m.locI_w);
  else k_locate<T, 3><<<nblocks(m.nm, 256), 256, 0, s>>>(m, m.X[0], m.X[1], m.X[2], m.locI_b, (T *)m.locI_w);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_interp(const MarkerArgs &m, const T *const u[3], cudaStream_t s) {
  if (m.nm == 0) return cudaSuccess;
  const unsigned g = nblocks((m.nm * m.dim + kInterpItems - 1) / kInterpItems * (m.dim == 3 ? 16 : 4), 256);
  if (m.dim == 2) return launch_pdl(k_interp<T, 2>, dim3(g), dim3(256), 0, s, m, u[0], u[1], u[1]);
  return launch_pdl(k_interp<T, 3>, dim3(g), dim3(256), 0, s, m, u[0], u[1], u[2]);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update(const MarkerArgs &m, cudaStream_t s) {
  if (m.nm == 0) return cudaSuccess;
  if (m.dim == 2) return launch_pdl(k_update<T, 2>, dim3(nblocks(m.nm * 2, kMarkerCta)), dim3(kMarkerCta), 0, s, m);
  return launch_pdl(k_update<T, 3>, dim3(nblocks(m.nm * 3, kMarkerCta)), dim3(kMarkerCta), 0, s, m);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_force(const MarkerArgs &m, cudaStream_t s) {
  if (m.nm == 0) return cudaSuccess;
  const unsigned g = nblocks(m.nm * 8, kMarkerCta);
  if (m.frac_force) {
    if (m.dim == 2) return launch_pdl(k_force<T, 2, true>, dim3(g), dim3(kMarkerCta), 0, s, m);
    return launch_pdl(k_force<T, 3, true>, dim3(g), dim3(kMarkerCta), 0, s, m);
  } else {
    if (m.dim == 2) return launch_pdl(k_force<T, 2, false>, dim3(g), dim3(kMarkerCta), 0, s, m);
    return launch_pdl(k_force<T, 3, false>, dim3(g), dim3(kMarkerCta), 0, s, m);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spread(const MarkerArgs &m, T *const f[3], cudaStream_t s) {
  if (m.nm == 0) return cudaSuccess;
  if (m.dim == 2)
    return launch_pdl(k_spread<T, 2>, dim3(nblocks(m.nm * 2 * 4, 256)), dim3(256), 0, s, m, f[0], f[1], f[1]);
  return launch_pdl(k_spread3<T>, dim3(nblocks((m.nm * 3 + kSpreadItems - 1) / kSpreadItems * 32, 256)), dim3(256), 0,
                    s, m, f[0], f[1], f[2]);
  return cudaGetLastError();
}

cudaError_t launch_markers_layout(double *aos, double *const X[3], const int32_t *perm, int64_t nm, int dim,
                                  int to_soa, cudaStream_t s) {
  if (nm == 0) return cudaSuccess;
  k_markers_layout<<<nblocks(nm * dim, 256), 256, 0, s>>>(aos, X[0], X[1], X[2], perm, nm, dim, to_soa);
  return cudaGetLastError();
}

// batched launchers: every member of the batch has the same dim and precision
template <typename T>
cudaError_t launch_interp_batch(const MarkerFieldArgs *a, int n, cudaStream_t s) {
  if (n < 1) return cudaSuccess;
  const int d = a[0].m.dim;
  std::vector<dim3> g(n);
  for (int i = 0; i < n; ++i)
    g[i] = dim3(a[i].m.nm ? nblocks((a[i].m.nm * d + kInterpItems - 1) / kInterpItems * (d == 3 ? 16 : 4), 256) : 0);
  if (d == 2) return launch_batch(k_interp_b<T, 2>, a, g.data(), n, dim3(256), s);
  return launch_batch(k_interp_b<T, 3>, a, g.data(), n, dim3(256), s);
}

template <typename T>
cudaError_t launch_update_batch(const MarkerArgs *m, int n, cudaStream_t s) {
  if (n < 1) return cudaSuccess;
  const int d = m[0].dim;
  std::vector<dim3> g(n);
  for (int i = 0; i < n; ++i) g[i] = dim3(m[i].nm ? nblocks(m[i].nm * d, kMarkerCta) : 0);
  if (d == 2) return launch_batch(k_update_b<T, 2>, m, g.data(), n, dim3(kMarkerCta), s);
  return launch_batch(k_update_b<T, 3>, m, g.data(), n, dim3(kMarkerCta), s);
}

template <typename T>
cudaError_t launch_force_batch(const MarkerArgs *m, int n, cudaStream_t s) {
  if (n < 1) return cudaSuccess;
  const int d = m[0].dim;
  std::vector<dim3> g(n);
  for (int i = 0; i < n; ++i) g[i] = dim3(m[i].nm ? nblocks(m[i].nm * 8, kMarkerCta) : 0);
  if (m[0].frac_force) {
    if (d == 2) return launch_batch(k_force_b<T, 2, true>, m, g.data(), n, dim3(kMarkerCta), s);
    return launch_batch(k_force_b<T, 3, true>, m, g.data(), n, dim3(kMarkerCta), s);
  }
  if (d == 2) return launch_batch(k_force_b<T, 2, false>, m, g.data(), n, dim3(kMarkerCta), s);
  return launch_batch(k_force_b<T, 3, false>, m, g.data(), n, dim3(kMarkerCta), s);
}

template <typename T>
cudaError_t launch_spread_batch(const MarkerFieldArgs *a, int n, cudaStream_t s) {
  if (n < 1) return cudaSuccess;
  const int d = a[0].m.dim;
  std::vector<dim3> g(n);
  for (int i = 0; i < n; ++i)
    g[i] = dim3(a[i].m.nm ? (d == 3 ? nblocks((a[i].m.nm * 3 + kSpreadItems - 1) / kSpreadItems * 32, 256)
                                    : nblocks(a[i].m.nm * 2 * 4, 256))
                          : 0);
  if (d == 2) return launch_batch(k_spread_b<T, 2>, a, g.data(), n, dim3(256), s);
  return launch_batch(k_spread3_b<T>, a, g.data(), n, dim3(256), s);
}

template cudaError_t launch_interp_batch<float>(const MarkerFieldArgs *, int, cudaStream_t);
template cudaError_t launch_interp_batch<double>(const MarkerFieldArgs *, int, cudaStream_t);
template cudaError_t launch_update_batch<float>(const MarkerArgs *, int, cudaStream_t);
template cudaError_t launch_update_batch<double>(const MarkerArgs *, int, cudaStream_t);
template cudaError_t launch_force_batch<float>(const MarkerArgs *, int, cudaStream_t);
template cudaError_t launch_force_batch<double>(const MarkerArgs *, int, cudaStream_t);
template cudaError_t launch_spread_batch<float>(const MarkerFieldArgs *, int, cudaStream_t);
template cudaError_t launch_spread_batch<double>(const MarkerFieldArgs *, int, cudaStream_t);

template cudaError_t launch_locate<float>(const MarkerArgs &, cudaStream_t);
template cudaError_t launch_locate<double>(const MarkerArgs &, cudaStream_t);
template cudaError_t launch_interp<float>(const MarkerArgs &, const float *const[3], cudaStream_t);
template cudaError_t launch_interp<double>(const MarkerArgs &, const double *const[3], cudaStream_t);
template cudaError_t launch_update<float>(const MarkerArgs &, cudaStream_t);
template cudaError_t launch_update<double>(const MarkerArgs &, cudaStream_t);
template cudaError_t launch_force<float>(const MarkerArgs &, cudaStream_t);
template cudaError_t launch_force<double>(const MarkerArgs &, cudaStream_t);
template cudaError_t launch_spread<float>(const MarkerArgs &, float *const[3], cudaStream_t);
template cudaError_t launch_spread<double>(const MarkerArgs &, double *const[3], cudaStream_t);

}  // namespace ibg
