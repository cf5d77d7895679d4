// Host runtime and C ABI of the sm_103a IB-GM step (include/ib_gb300.h).
//
// One ib_grid_t owns, on the current device:
//   fields  (precision T): u[d], p, psi, Nold[d] = N(u^{n-1}), div = D.u^n,
//           scr[d] (momentum increment R, to which spreading adds dt/rho f,
//           then the sweep results), all in one allocation;
//   markers (FP64 SoA): X, Xh = X^{n+1/2}, U = U^n, Uold = U^{n-1}, G, plus
//           the force connections as CSR by marker and as an edge list;
//   line-solve tables: lam^k (k = 0..n_a) per axis for the momentum operator
//           (r = mu dt / (2 rho h_a^2)) and the psi operator (r = 1 / h_a^2).
// A step is 11 launches in 3D (9 in 2D): interp, update, force, rhs, spread,
// d momentum sweeps, d psi sweeps.
// Steps after the first replay a CUDA graph (one per split-order phase) on a
// library-owned stream that is ordered against the caller's stream with
// events.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/ib_gb300.h"
#include "ib_internal.cuh"

using namespace ibg;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define IB_CUDA(call)                                                                               \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return fail(IB_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
  } while (0)

// lam, c and lam^k of the cyclic operator (1 + 2r) I - r (S + S^{-1}) =
// c (I - lam S)(I - lam S^{-1}); computed in FP64 on the host.
struct HostCoef {
  double lam, inv_c, inv_1m;
  std::vector<double> pw;
};
HostCoef make_coef(int n, double r) {
  HostCoef h;
  const double lam = 2.0 * r / (1.0 + 2.0 * r + sqrt(1.0 + 4.0 * r));
  h.lam = lam;
  h.inv_c = 2.0 / (1.0 + 2.0 * r + sqrt(1.0 + 4.0 * r));  // 1 / c, c = r / lam
  h.pw.resize(n + 1);
  double p = 1.0;
  for (int k = 0; k <= n; ++k) {
    h.pw[k] = p;
    p *= lam;
  }
  h.inv_1m = 1.0 / (1.0 - h.pw[n]);
  return h;
}

// device copy of a coefficient table in both precisions
struct DevCoef {
  void *mem = nullptr;
  LineCoef<float> f;
  LineCoef<double> d;
};
int upload_coef(const HostCoef &h, DevCoef &out, cudaStream_t s) {
  const int m = (int)h.pw.size();
  size_t bytes = m * sizeof(double) + 2 * m * sizeof(float) + 64;
  IB_CUDA(cudaMalloc(&out.mem, bytes));
  double *pd = (double *)out.mem;
  float *pf = (float *)(pd + m);
  float *pf_lo = pf + m;
  // FP32 tables: lam^k rounded, and the remainder lam^k - (float)lam^k
  std::vector<float> hf(2 * m);
  for (int k = 0; k < m; ++k) {
    hf[k] = (float)h.pw[k];
    hf[m + k] = (float)(h.pw[k] - (double)hf[k]);
  }
  IB_CUDA(cudaMemcpyAsync(pd, h.pw.data(), m * sizeof(double), cudaMemcpyHostToDevice, s));
  IB_CUDA(cudaMemcpyAsync(pf, hf.data(), 2 * m * sizeof(float), cudaMemcpyHostToDevice, s));
  IB_CUDA(cudaStreamSynchronize(s));
  out.d = LineCoef<double>{pd, h.lam, h.inv_c, h.inv_1m, nullptr, 0.0, 0};
  // FP32 solves evaluate the periodic correction to FP64 accuracy whenever
  // the wrap weight lam^n is above FP32 resolution
  const int ext = h.pw[m - 1] > 0x1p-24 ? 1 : 0;
  const float q_hi = (float)h.inv_1m;
  out.f = LineCoef<float>{pf, (float)h.lam, (float)h.inv_c, q_hi, pf_lo, (float)(h.inv_1m - (double)q_hi), ext};
  return IB_OK;
}

template <typename T>
const LineCoef<T> &coef_of(const DevCoef &c);
template <>
const LineCoef<float> &coef_of<float>(const DevCoef &c) { return c.f; }
template <>
const LineCoef<double> &coef_of<double>(const DevCoef &c) { return c.d; }

// Coefficients of sweep st of a chain of d sweeps over the operators co[ax]:
// the sweeps are linear, so the chain applies the product of its 1/c once,
// in the last sweep, and the others run unscaled.
constexpr int kAxes[3] = {0, 1, 2};
template <typename T>
LineCoef<T> chain_coef(const DevCoef *co, const int *order, int st, int d) {
  LineCoef<T> c = coef_of<T>(co[order[st]]);
  double prod = 1.0;
  for (int q = 0; q < d; ++q) prod *= co[order[q]].d.scale;
  c.scale = st == d - 1 ? (T)prod : T(1);
  return c;
}

// process-wide cache for the stand-alone line-solve entry points
std::mutex g_cache_mu;
std::map<std::tuple<int, int, double>, DevCoef> g_cache;  // (device, n, r)

int cached_coef(int n, double r, cudaStream_t s, DevCoef **out) {
  int dev = 0;
  IB_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto key = std::make_tuple(dev, n, r);
  auto it = g_cache.find(key);
  if (it == g_cache.end()) {
    DevCoef c;
    cudaStream_t tmp;
    IB_CUDA(cudaStreamCreateWithFlags(&tmp, cudaStreamNonBlocking));
    int rc = upload_coef(make_coef(n, r), c, tmp);
    cudaStreamDestroy(tmp);
    if (rc != IB_OK) return rc;
    it = g_cache.emplace(key, c).first;
  }
  *out = &it->second;
  (void)s;
  return IB_OK;
}

}  // namespace

const char *ib_kernel_name(int slot);

// error recording for the other translation units of the library
int ib_internal_fail(int code, const char *msg) { return fail(code, "%s", msg); }

struct ib_grid_s {
  ib_grid_desc desc;
  int dim = 0, prec = 0;
  int n[3] = {1, 1, 1};
  long long cells = 0;
  double h[3] = {1, 1, 1};
  size_t esz = 4;
  void *fields = nullptr;
  void *u[3] = {}, *p = nullptr, *psi = nullptr, *Nold[3] = {}, *div = nullptr, *scr[3] = {};
  DevCoef coef[2][3];  // [0: momentum, 1: psi][axis]

  // markers
  std::vector<double> hX;       // [nm][dim]
  std::vector<int32_t> hE;      // [ne][2] global indices
  std::vector<double> hK, hR;   // [ne]
  std::vector<int32_t> hT;      // [nt][3] global indices
  int64_t nm = 0, ne = 0, nt = 0;
  int nfibers = 0;
  bool markers_uploaded = false;
  void *mk = nullptr;           // one allocation for all marker data
  double *X[3] = {}, *Xh[3] = {};
  void *U[3] = {}, *Uold[3] = {}, *G[3] = {};  // field precision
  int32_t *locI_b = nullptr, *locS_b = nullptr;  // [2d][nm] grid locations (see MarkerArgs)
  void *locI_w = nullptr, *locS_w = nullptr;      // [2d][nm][4] their weights
  void *locS_f = nullptr;       // [d][nm] own-axis fraction of X^{n+1/2}
  void *kapT = nullptr, *restT = nullptr;  // [2ne] CSR spring data in the field precision
  int64_t *row = nullptr;
  int32_t *col = nullptr, *edges = nullptr, *tris = nullptr;
  double *kap = nullptr, *rest = nullptr, *ekap = nullptr, *erest = nullptr;
  double *acc = nullptr;        // diagnostics accumulators (device)
  double *stage = nullptr;      // [nm][dim] staging buffer for marker I/O
  int32_t *perm = nullptr;      // internal marker k is the caller's marker perm[k]
  int32_t *cedge = nullptr;     // connection index of every CSR entry

  int64_t step = 0;
  bool div_valid = false;
  bool loc_valid = false;       // locI holds the grid locations of the current X
  bool tuned = false;
  int tune[3] = {-1, -1, -1};   // sweep configuration per axis (autotuned)
  int tune_r[3] = {-1, -1, -1}; // the best one for the sweeps with a prologue or epilogue (no TMA kernel)
  int tune_psi[3] = {-1, -1, -1};  // plain psi sweeps (one field, the psi operator)
  int tune_div[3] = {-1, -1, -1};  // the first psi sweep (divergence prologue; no TMA kernel)
  int tune_addu[3] = {-1, -1, -1}; // the last momentum sweep (u^n + e epilogue; no TMA kernel)
  int tune_p[3] = {-1, -1, -1};    // the last psi sweep (p + psi epilogue; no TMA kernel)
  bool fixed[3] = {false, false, false};  // set by ib_fix_sweep_config: not timed
  int resort_every = 0;         // ib_set_resort_interval: re-sort the markers every that many steps
  cudaStream_t s = nullptr;     // library stream
  cudaStream_t user = nullptr;  // caller stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaStream_t s2 = nullptr;    // marker branch of a step (interp, update, force beside the rhs)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
};

namespace {

MarkerArgs marker_args(ib_grid_s *g, bool first) {
  const int d = g->dim;
  MarkerArgs m;
  memset(&m, 0, sizeof(m));
  for (int a = 0; a < 3; ++a) {
    m.X[a] = g->X[a];
    m.Xh[a] = g->Xh[a];
    m.U[a] = g->U[a];
    m.Uold[a] = g->Uold[a];
    m.G[a] = g->G[a];
    m.inv_h[a] = 1.0 / g->h[a];
    m.n[a] = g->n[a];
  }
  m.locI_b = g->locI_b;
  m.locI_w = g->locI_w;
  m.locS_b = g->locS_b;
  m.locS_w = g->locS_w;
  m.locS_f = g->locS_f;
  m.kapT = g->kapT;
  m.restT = g->restT;
  for (int a = 0; a < 3; ++a) {
    m.h32[a] = (float)g->h[a];
    m.inv_n32[a] = 1.0f / (float)g->n[a];
  }
  m.frac_force = g->prec == IB_FP32 ? 1 : 0;
  m.row = g->row;
  m.col = g->col;
  m.kap = g->kap;
  m.rest = g->rest;
  m.nm = g->nm;
  m.dt = g->desc.dt;
  m.H = g->desc.H;
  m.spread_scale = g->desc.dt / g->desc.rho;
  for (int a = 0; a < d; ++a) m.spread_scale /= g->h[a];
  m.dim = d;
  m.kernel = g->desc.kernel;
  m.first = first ? 1 : 0;
  return m;
}

// The arguments of every kernel of one step (Sec. 3.4, Steps 1a-3f) of grid
// g: the marker chain, the right-hand side, spreading and the 2d sweeps with
// their configurations.  enqueue_step_t launches one plan; an ensemble
// launches the plans of a size class together (batched launches).
template <typename T>
struct StepPlan {
  MarkerArgs m;
  const T *uc[3];
  T *sc[3];
  RhsArgs<T> ra;
  SweepArgs<T> sw[6];
  int ax[6], pro[6], epi[6], nf[6], cfg[6], cfg_r[6];
  int nsw;
};

template <typename T>
void plan_step(ib_grid_s *g, bool first, int phase, StepPlan<T> &P) {
  const int d = g->dim;
  int order[3];
  for (int i = 0; i < d; ++i) order[i] = (i + phase) % d;
  P.m = marker_args(g, first);
  for (int a = 0; a < 3; ++a) {
    P.uc[a] = (const T *)g->u[a];
    P.sc[a] = (T *)g->scr[a];
  }
  // Steps 3a-3b
  RhsArgs<T> &ra = P.ra;
  memset(&ra, 0, sizeof(ra));
  for (int a = 0; a < 3; ++a) {
    ra.u[a] = P.uc[a];
    ra.Nold[a] = (T *)g->Nold[a];
    ra.scr[a] = P.sc[a];
    ra.inv_h[a] = (T)(1.0 / g->h[a]);
    ra.inv_h2[a] = (T)(1.0 / (g->h[a] * g->h[a]));
    ra.n[a] = g->n[a];
  }
  {
    const double dt = g->desc.dt, rho = g->desc.rho;
    ra.cmu = (T)(dt * g->desc.mu / rho);
    for (int a = 0; a < 3; ++a) ra.ncg[a] = (T)(-dt / (rho * g->h[a]));
    ra.ncA = (T)(first ? -dt : -1.5 * dt);
    ra.cN = (T)(first ? 0.0 : 0.5 * dt);
  }
  const bool gm1 = g->desc.scheme == IB_GM1;
  ra.p = (const T *)g->p;
  ra.psi = gm1 ? nullptr : (const T *)g->psi;
  ra.first = first ? 1 : 0;
  // Steps 3c-3d (+ z): increment-form Douglas sweeps on the scratch fields
  SweepArgs<T> sa;
  memset(&sa, 0, sizeof(sa));
  for (int a = 0; a < 3; ++a) {
    sa.f[a] = P.sc[a];
    sa.u[a] = P.uc[a];
    sa.uo[a] = (T *)g->u[a];
    sa.inv_h[a] = (T)(1.0 / g->h[a]);
    sa.n[a] = g->n[a];
  }
  sa.p = (T *)g->p;
  sa.div = (T *)g->div;
  sa.pro_scale = (T)(-g->desc.rho / g->desc.dt);
  sa.chi_mu_half = gm1 ? T(0) : (T)(0.5 * g->desc.chi * g->desc.mu);
  sa.p_keep = gm1 ? T(0) : T(1);
  sa.dim = d;
  int k = 0;
  for (int st = 0; st < d; ++st, ++k) {
    const int ax = order[st];
    sa.co = chain_coef<T>(g->coef[0], order, st, d);
    const bool last = st == d - 1;
    P.sw[k] = sa;
    P.ax[k] = ax;
    P.pro[k] = PRO_LOAD;
    P.epi[k] = last ? EPI_ADDU : EPI_STORE;
    P.nf[k] = d;
    P.cfg[k] = last ? g->tune_addu[ax] : g->tune[ax];
    P.cfg_r[k] = last ? g->tune_addu[ax] : g->tune_r[ax];
  }
  // Step 3e (psi, one sweep per axis) with Step 3f folded into the first and
  // last sweeps
  sa.f[0] = sa.f[1] = sa.f[2] = (T *)g->psi;
  for (int st = 0; st < d; ++st, ++k) {
    const int ax = order[st];
    sa.co = chain_coef<T>(g->coef[1], order, st, d);
    const int pro = st == 0 ? PRO_DIV : PRO_LOAD;
    const int epi = st == d - 1 ? EPI_P : EPI_STORE;
    const bool plain = pro == PRO_LOAD && epi == EPI_STORE;
    P.sw[k] = sa;
    P.ax[k] = ax;
    P.pro[k] = pro;
    P.epi[k] = epi;
    P.nf[k] = 1;
    P.cfg[k] = pro == PRO_DIV ? g->tune_div[ax] : plain ? g->tune_psi[ax] : g->tune_p[ax];
    P.cfg_r[k] = pro == PRO_DIV ? g->tune_div[ax] : plain ? g->tune_r[ax] : g->tune_p[ax];
  }
  P.nsw = k;
}

template <typename T>
int enqueue_step_t(ib_grid_s *g, bool first, int phase, cudaEvent_t *ev) {
  auto mark = [&](int slot) -> int {
    if (ev) IB_CUDA(cudaEventRecord(ev[slot], g->s));
    return IB_OK;
  };
  int rc;
  StepPlan<T> P;
  plan_step<T>(g, first, phase, P);
  // Steps 1a-2a; spreading (Step 2b) follows the right-hand side, into which
  // it adds dt/rho f
  // the marker chain (interp, update, force) runs on a second, higher-priority
  // stream beside the right-hand side (they share no data); spreading waits
  // for both.  Profiling (ev set) keeps one stream so that every kernel is
  // timed alone.
  const bool fork = !ev && g->nm > 0;
  if ((rc = mark(0))) return rc;
  cudaStream_t ms = g->s;
  if (fork) {
    IB_CUDA(cudaEventRecord(g->ev_fork, g->s));
    IB_CUDA(cudaStreamWaitEvent(g->s2, g->ev_fork, 0));
    ms = g->s2;
  }
  IB_CUDA(launch_interp<T>(P.m, P.uc, ms));
  if ((rc = mark(1))) return rc;
  IB_CUDA(launch_update<T>(P.m, ms));
  if ((rc = mark(2))) return rc;
  IB_CUDA(launch_force<T>(P.m, ms));
  if ((rc = mark(3))) return rc;
  if (fork) IB_CUDA(cudaEventRecord(g->ev_join, g->s2));
  // Steps 3a-3b
  IB_CUDA(launch_rhs<T>(g->dim, P.ra, g->s));
  if ((rc = mark(4))) return rc;
  if (fork) IB_CUDA(cudaStreamWaitEvent(g->s, g->ev_join, 0));
  // Step 2b: R += dt/rho S(X^{n+1/2}) G
  IB_CUDA(launch_spread<T>(P.m, P.sc, g->s));
  if ((rc = mark(5))) return rc;
  // Steps 3c-3f: marks 6 + s after the s-th momentum sweep, 9 + s after the
  // s-th psi sweep
  for (int k = 0; k < P.nsw; ++k) {
    IB_CUDA(launch_sweep<T>(P.ax[k], P.pro[k], P.epi[k], P.nf[k], P.sw[k], g->s, P.cfg[k]));
    if ((rc = mark(k < g->dim ? 6 + k : 9 + (k - g->dim)))) return rc;
  }
  return IB_OK;
}

int enqueue_step(ib_grid_s *g, bool first, int phase, cudaEvent_t *ev) {
  return g->prec == IB_FP32 ? enqueue_step_t<float>(g, first, phase, ev)
                            : enqueue_step_t<double>(g, first, phase, ev);
}

int ensure_div(ib_grid_s *g) {
  if (g->div_valid) return IB_OK;
  if (g->prec == IB_FP32) {
    const float *uc[3] = {(const float *)g->u[0], (const float *)g->u[1], (const float *)g->u[2]};
    const float ih[3] = {(float)(1.0 / g->h[0]), (float)(1.0 / g->h[1]), (float)(1.0 / g->h[2])};
    IB_CUDA(launch_divergence<float>(g->dim, uc, (float *)g->div, g->n, ih, g->s));
  } else {
    const double *uc[3] = {(const double *)g->u[0], (const double *)g->u[1], (const double *)g->u[2]};
    const double ih[3] = {1.0 / g->h[0], 1.0 / g->h[1], 1.0 / g->h[2]};
    IB_CUDA(launch_divergence<double>(g->dim, uc, (double *)g->div, g->n, ih, g->s));
  }
  g->div_valid = true;
  return IB_OK;
}

// Build the device marker arrays and the CSR neighbour lists (once, before the
// first step).
// Interleave the low 10 bits of up to three cell coordinates (Morton order).
uint64_t morton_key(const unsigned q[3], int d) {
  uint64_t key = 0;
  for (int bit = 9; bit >= 0; --bit)
    for (int a = d - 1; a >= 0; --a) key = (key << 1) | ((q[a] >> bit) & 1u);
  return key;
}

// Morton order of nm positions (component a of marker k at X[k * sk + a * sa])
// wrapped into the box: order[i] = index of the i-th marker in that order
void morton_order(const double *X, int64_t nm, int d, double H, int64_t sk, int64_t sa, std::vector<int32_t> &order) {
  std::vector<uint64_t> key(nm);
  for (int64_t k = 0; k < nm; ++k) {
    unsigned q[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
      double x = X[k * sk + a * sa] / H;
      x -= floor(x);
      int c = (int)(x * 1024.0);
      q[a] = (unsigned)(c < 0 ? 0 : (c > 1023 ? 1023 : c));
    }
    key[k] = morton_key(q, d);
  }
  order.resize(nm);
  for (int64_t k = 0; k < nm; ++k) order[k] = (int32_t)k;
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return key[x] < key[y]; });
}

// The structure arrays of the internal marker numbering perm (perm[k] =
// caller's index of internal marker k): connections as CSR by marker (both
// directions) and as an edge list, triangles, and perm itself, written into
// the grid's existing device buffers.
int upload_structure(ib_grid_s *g, const std::vector<int32_t> &perm) {
  const int64_t nm = g->nm, ne = g->ne, nt = g->nt;
  std::vector<int32_t> inv(nm);
  for (int64_t k = 0; k < nm; ++k) inv[perm[k]] = (int32_t)k;
  std::vector<int32_t> E(2 * ne), Tr(3 * nt);
  for (int64_t e = 0; e < 2 * ne; ++e) E[e] = inv[g->hE[e]];
  for (int64_t t = 0; t < 3 * nt; ++t) Tr[t] = inv[g->hT[t]];
  std::vector<int64_t> row(nm + 1, 0);
  for (int64_t e = 0; e < ne; ++e) {
    row[E[2 * e] + 1]++;
    row[E[2 * e + 1] + 1]++;
  }
  for (int64_t a = 0; a < nm; ++a) row[a + 1] += row[a];
  std::vector<int32_t> col(2 * ne), cedge(2 * ne);
  std::vector<double> kap(2 * ne), rest(2 * ne);
  std::vector<float> kapf(g->esz == 4 ? 2 * ne : 0), restf(g->esz == 4 ? 2 * ne : 0);
  std::vector<int64_t> fill(row.begin(), row.end() - 1);
  for (int64_t e = 0; e < ne; ++e) {
    const int32_t a = E[2 * e], b = E[2 * e + 1];
    int64_t pa = fill[a]++, pb = fill[b]++;
    col[pa] = b;
    col[pb] = a;
    cedge[pa] = cedge[pb] = (int32_t)e;
    kap[pa] = kap[pb] = g->hK[e];
    rest[pa] = rest[pb] = g->hR[e];
  }
  IB_CUDA(cudaMemcpyAsync(g->row, row.data(), sizeof(int64_t) * (nm + 1), cudaMemcpyHostToDevice, g->s));
  if (ne) {
    IB_CUDA(cudaMemcpyAsync(g->col, col.data(), sizeof(int32_t) * 2 * ne, cudaMemcpyHostToDevice, g->s));
    IB_CUDA(cudaMemcpyAsync(g->cedge, cedge.data(), sizeof(int32_t) * 2 * ne, cudaMemcpyHostToDevice, g->s));
    IB_CUDA(cudaMemcpyAsync(g->kap, kap.data(), sizeof(double) * 2 * ne, cudaMemcpyHostToDevice, g->s));
    IB_CUDA(cudaMemcpyAsync(g->rest, rest.data(), sizeof(double) * 2 * ne, cudaMemcpyHostToDevice, g->s));
    if (g->esz == 4) {
      for (int64_t e = 0; e < 2 * ne; ++e) {
        kapf[e] = (float)kap[e];
        restf[e] = (float)rest[e];
      }
      IB_CUDA(cudaMemcpyAsync(g->kapT, kapf.data(), sizeof(float) * 2 * ne, cudaMemcpyHostToDevice, g->s));
      IB_CUDA(cudaMemcpyAsync(g->restT, restf.data(), sizeof(float) * 2 * ne, cudaMemcpyHostToDevice, g->s));
    } else {
      IB_CUDA(cudaMemcpyAsync(g->kapT, kap.data(), sizeof(double) * 2 * ne, cudaMemcpyHostToDevice, g->s));
      IB_CUDA(cudaMemcpyAsync(g->restT, rest.data(), sizeof(double) * 2 * ne, cudaMemcpyHostToDevice, g->s));
    }
    IB_CUDA(cudaMemcpyAsync(g->edges, E.data(), sizeof(int32_t) * 2 * ne, cudaMemcpyHostToDevice, g->s));
  }
  if (nt) IB_CUDA(cudaMemcpyAsync(g->tris, Tr.data(), sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice, g->s));
  if (nm) IB_CUDA(cudaMemcpyAsync(g->perm, perm.data(), sizeof(int32_t) * nm, cudaMemcpyHostToDevice, g->s));
  IB_CUDA(cudaStreamSynchronize(g->s));  // host vectors above go out of scope
  return IB_OK;
}

int upload_markers(ib_grid_s *g) {
  if (g->markers_uploaded) return IB_OK;
  const int d = g->dim;
  const int64_t nm = g->nm, ne = g->ne, nt = g->nt;
  // Internal marker order: Morton order of the initial positions (wrapped into
  // the box), so that runs of consecutive markers are spatially compact.
  // perm[k] = caller's index of internal marker k.
  std::vector<int32_t> perm;
  morton_order(g->hX.data(), nm, d, g->desc.H, d, 1, perm);
  std::vector<double> soa(nm * d);
  for (int64_t k = 0; k < nm; ++k)
    for (int a = 0; a < d; ++a) soa[a * nm + k] = g->hX[(int64_t)perm[k] * d + a];
  // layout: X, Xh (FP64) | U, Uold, G (field precision) | row | col | kap |
  // rest | edges | ekap | erest | tris | acc | stage | perm | locations
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  const size_t es = g->esz;
  const size_t o_m = take(sizeof(double) * 2 * d * (nm + 1));
  const size_t o_u = take(es * 3 * d * (nm + 1));
  const size_t o_row = take(sizeof(int64_t) * (nm + 1));
  const size_t o_col = take(sizeof(int32_t) * (2 * ne + 1));
  const size_t o_kap = take(sizeof(double) * (2 * ne + 1));
  const size_t o_rest = take(sizeof(double) * (2 * ne + 1));
  const size_t o_e = take(sizeof(int32_t) * (2 * ne + 1));
  const size_t o_ek = take(sizeof(double) * (ne + 1));
  const size_t o_er = take(sizeof(double) * (ne + 1));
  const size_t o_t = take(sizeof(int32_t) * (3 * nt + 1));
  const size_t o_acc = take(sizeof(double) * 8);
  const size_t o_stage = take(sizeof(double) * (nm * d + 1));
  const size_t o_perm = take(sizeof(int32_t) * (nm + 1));
  const size_t o_cedge = take(sizeof(int32_t) * (2 * ne + 1));
  const size_t o_lib = take(sizeof(int32_t) * 2 * d * (nm + 1));
  const size_t o_lsb = take(sizeof(int32_t) * 2 * d * (nm + 1));
  const size_t o_lif = take(es * 4 * 2 * d * (nm + 1));
  const size_t o_lsf = take(es * 4 * 2 * d * (nm + 1));
  const size_t o_lff = take(es * d * (nm + 1));
  const size_t o_kt = take(es * (2 * ne + 1));
  const size_t o_rt = take(es * (2 * ne + 1));
  if (cudaMalloc(&g->mk, off) != cudaSuccess) return fail(IB_ERR_OOM, "marker allocation of %zu bytes failed", off);
  char *base = (char *)g->mk;
  double *md = (double *)(base + o_m);
  char *mu = base + o_u;
  for (int a = 0; a < 3; ++a) {
    const int aa = a < d ? a : d - 1;
    g->X[a] = md + (0 * d + aa) * nm;
    g->Xh[a] = md + (1 * d + aa) * nm;
    g->U[a] = mu + es * (0 * d + aa) * nm;
    g->Uold[a] = mu + es * (1 * d + aa) * nm;
    g->G[a] = mu + es * (2 * d + aa) * nm;
  }
  g->locI_b = (int32_t *)(base + o_lib);
  g->locS_b = (int32_t *)(base + o_lsb);
  g->locI_w = base + o_lif;
  g->locS_w = base + o_lsf;
  g->locS_f = base + o_lff;
  g->kapT = base + o_kt;
  g->restT = base + o_rt;
  g->row = (int64_t *)(base + o_row);
  g->col = (int32_t *)(base + o_col);
  g->kap = (double *)(base + o_kap);
  g->rest = (double *)(base + o_rest);
  g->edges = (int32_t *)(base + o_e);
  g->ekap = (double *)(base + o_ek);
  g->erest = (double *)(base + o_er);
  g->tris = (int32_t *)(base + o_t);
  g->acc = (double *)(base + o_acc);
  g->stage = (double *)(base + o_stage);
  g->perm = (int32_t *)(base + o_perm);
  g->cedge = (int32_t *)(base + o_cedge);
  IB_CUDA(cudaMemsetAsync(g->mk, 0, off, g->s));
  if (nm) IB_CUDA(cudaMemcpyAsync(g->X[0], soa.data(), sizeof(double) * nm * d, cudaMemcpyHostToDevice, g->s));
  if (ne) {
    IB_CUDA(cudaMemcpyAsync(g->ekap, g->hK.data(), sizeof(double) * ne, cudaMemcpyHostToDevice, g->s));
    IB_CUDA(cudaMemcpyAsync(g->erest, g->hR.data(), sizeof(double) * ne, cudaMemcpyHostToDevice, g->s));
  }
  int rc = upload_structure(g, perm);  // synchronises the stream (soa goes out of scope)
  if (rc) return rc;
  g->markers_uploaded = true;
  return IB_OK;
}

int enter(ib_grid_s *g) {
  IB_CUDA(cudaEventRecord(g->ev_in, g->user));
  IB_CUDA(cudaStreamWaitEvent(g->s, g->ev_in, 0));
  return IB_OK;
}
int leave(ib_grid_s *g) {
  IB_CUDA(cudaEventRecord(g->ev_out, g->s));
  IB_CUDA(cudaStreamWaitEvent(g->user, g->ev_out, 0));
  return IB_OK;
}

int get_graph(ib_grid_s *g, int phase) {
  if (g->graph[phase]) return IB_OK;
  cudaGraph_t graph;
  IB_CUDA(cudaStreamBeginCapture(g->s, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_step(g, false, phase, nullptr);
  cudaError_t e = cudaStreamEndCapture(g->s, &graph);
  if (rc != IB_OK) {
    if (e == cudaSuccess) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return fail(IB_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&g->graph[phase], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(IB_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return IB_OK;
}

int ensure_loc(ib_grid_s *g) {
  if (g->loc_valid) return IB_OK;
  const MarkerArgs m = marker_args(g, false);
  IB_CUDA(g->prec == IB_FP32 ? launch_locate<float>(m, g->s) : launch_locate<double>(m, g->s));
  g->loc_valid = true;
  return IB_OK;
}

// Autotuner: for every axis, time each candidate sweep configuration in the
// five roles the step uses it in, 1 + 3 launches each, and keep the fastest
// per role: the plain momentum sweep on the d scratch fields (tune; tune_r,
// the best register kernel, serves the ensembles' batched plain sweeps), the
// last momentum sweep with its u^n + e epilogue (tune_addu; u^n is the
// scratch field itself, which every thread reads before it writes), the
// plain psi sweep on one scratch field with the psi operator (tune_psi), the
// first psi sweep with its divergence prologue (tune_div), which reads the
// state's velocity and writes D.u and p into two temporary fields, and the
// last psi sweep with its p + psi epilogue (tune_p, p in a temporary field).
// The sweeps with a prologue or epilogue have no TMA form.
template <typename T>
int autotune_t(ib_grid_s *g) {
  const int d = g->dim;
  SweepArgs<T> sa;
  memset(&sa, 0, sizeof(sa));
  for (int a = 0; a < 3; ++a) {
    sa.f[a] = (T *)g->scr[a];
    sa.n[a] = g->n[a];
    sa.inv_h[a] = (T)(1.0 / g->h[a]);
  }
  sa.dim = d;
  const size_t fb = ((size_t)g->cells * g->esz + 255) / 256 * 256;
  char *tmp = nullptr;
  if (cudaMalloc(&tmp, 2 * fb) != cudaSuccess) return fail(IB_ERR_OOM, "autotune scratch of %zu bytes", 2 * fb);
  SweepArgs<T> sd = sa;
  for (int a = 0; a < 3; ++a) sd.u[a] = (const T *)g->u[a < d ? a : 0];
  sd.f[0] = (T *)g->scr[0];
  sd.div = (T *)tmp;
  sd.p = (T *)(tmp + fb);
  sd.pro_scale = T(1);
  sd.p_keep = T(1);
  SweepArgs<T> su = sa;  // u^n + e into the scratch fields themselves
  for (int a = 0; a < 3; ++a) su.uo[a] = (T *)g->scr[a];
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = IB_OK;
  if (cudaMemsetAsync(tmp, 0, 2 * fb, g->s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    rc = fail(IB_ERR_CUDA, "autotune setup");
  // ms of 3 launches after one untimed launch, or < 0 on failure
  auto time = [&](int ax, int pro, int epi, int nf, const SweepArgs<T> &a, int cfg) -> float {
    if (launch_sweep<T>(ax, pro, epi, nf, a, g->s, cfg) != cudaSuccess) return -1.f;
    cudaEventRecord(e0, g->s);
    for (int r = 0; r < 3; ++r) launch_sweep<T>(ax, pro, epi, nf, a, g->s, cfg);
    cudaEventRecord(e1, g->s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  for (int ax = 0; ax < d && !rc; ++ax) {
    if (g->fixed[ax]) continue;
    sa.co = coef_of<T>(g->coef[0][ax]);
    su.co = sa.co;
    SweepArgs<T> sp = sa;
    sp.co = coef_of<T>(g->coef[1][ax]);
    sd.co = sp.co;
    int cand[24];
    const int nc = sweep_candidates(ax, g->n[ax], g->n[0], sizeof(T) == 8, cand, 24);
    float best = 1e30f, best_r = 1e30f, best_p = 1e30f, best_d = 1e30f, best_u = 1e30f, best_e = 1e30f;
    for (int i = 0; i < nc && !rc; ++i) {
      const bool reg = cand[i] != kTmaCfg;
      float t[5];
      t[0] = time(ax, PRO_LOAD, EPI_STORE, d, sa, cand[i]);
      t[1] = t[0] < 0.f ? t[0] : time(ax, PRO_LOAD, EPI_STORE, 1, sp, cand[i]);
      t[2] = t[1] < 0.f || !reg ? t[1] : time(ax, PRO_DIV, EPI_STORE, 1, sd, cand[i]);
      t[3] = t[2] < 0.f || !reg ? t[2] : time(ax, PRO_LOAD, EPI_ADDU, d, su, cand[i]);
      t[4] = t[3] < 0.f || !reg ? t[3] : time(ax, PRO_LOAD, EPI_P, 1, sd, cand[i]);
      if (t[0] < 0.f || t[1] < 0.f || t[2] < 0.f || t[3] < 0.f || t[4] < 0.f) {
        rc = fail(IB_ERR_CUDA, "autotune launch");
        break;
      }
      auto keep = [&](float ms, float &b, int *slot) {
        if (ms < b) {
          b = ms;
          slot[ax] = cand[i];
        }
      };
      keep(t[0], best, g->tune);
      keep(t[1], best_p, g->tune_psi);
      if (reg) {
        keep(t[0], best_r, g->tune_r);
        keep(t[2], best_d, g->tune_div);
        keep(t[3], best_u, g->tune_addu);
        keep(t[4], best_e, g->tune_p);
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(g->s);
  cudaFree(tmp);
  return rc;
}

int autotune(ib_grid_s *g) {
  if (g->tuned) return IB_OK;
  int rc = g->prec == IB_FP32 ? autotune_t<float>(g) : autotune_t<double>(g);
  g->tuned = true;
  return rc;
}

int prepare(ib_grid_s *g) {
  int rc = upload_markers(g);
  if (rc) return rc;
  if ((rc = ensure_loc(g))) return rc;
  if ((rc = ensure_div(g))) return rc;
  if ((rc = autotune(g))) return rc;
  // capture the step graph of every split-order phase up front so that no
  // instantiation happens between later steps
  const int phases = g->desc.rotate_split ? g->dim : 1;
  for (int ph = 0; ph < phases; ++ph)
    if ((rc = get_graph(g, ph))) return rc;
  return IB_OK;
}

// Re-number the markers internally in the Morton order of their current
// positions: X^n and U^{n-1} are permuted, the connection CSR, edge list,
// triangles and the caller permutation rebuilt, and the grid locations of X^n
// recomputed; every other marker array is rewritten by the next step before
// it is read.  Pointers do not change, so captured graphs stay valid.
// Synchronises the grid's stream.
int resort_markers(ib_grid_s *g) {
  if (!g->markers_uploaded || g->nm == 0) return IB_OK;
  const int d = g->dim;
  const int64_t nm = g->nm;
  const size_t es = g->esz;
  std::vector<double> X(nm * d), X2(nm * d);
  std::vector<char> Uo(es * nm * d), Uo2(es * nm * d);
  std::vector<int32_t> perm(nm), perm2(nm), ord;
  IB_CUDA(cudaMemcpyAsync(X.data(), g->X[0], sizeof(double) * nm * d, cudaMemcpyDeviceToHost, g->s));
  IB_CUDA(cudaMemcpyAsync(Uo.data(), g->Uold[0], es * nm * d, cudaMemcpyDeviceToHost, g->s));
  IB_CUDA(cudaMemcpyAsync(perm.data(), g->perm, sizeof(int32_t) * nm, cudaMemcpyDeviceToHost, g->s));
  IB_CUDA(cudaStreamSynchronize(g->s));
  morton_order(X.data(), nm, d, g->desc.H, 1, nm, ord);
  for (int64_t k = 0; k < nm; ++k) {
    perm2[k] = perm[ord[k]];
    for (int a = 0; a < d; ++a) {
      X2[a * nm + k] = X[a * nm + ord[k]];
      memcpy(Uo2.data() + es * (a * nm + k), Uo.data() + es * (a * nm + ord[k]), es);
    }
  }
  IB_CUDA(cudaMemcpyAsync(g->X[0], X2.data(), sizeof(double) * nm * d, cudaMemcpyHostToDevice, g->s));
  IB_CUDA(cudaMemcpyAsync(g->Uold[0], Uo2.data(), es * nm * d, cudaMemcpyHostToDevice, g->s));
  int rc = upload_structure(g, perm2);  // synchronises the stream
  if (rc) return rc;
  g->loc_valid = false;
  return ensure_loc(g);
}

// ---------------------------------------------------------------------------
// Discrete adjoint driver (kernels in ib_adjoint.cu).

// One forward step of the grid's own path (the body of ib_step's loop).
int forward_one(ib_grid_s *g) {
  int rc;
  if (g->step == 0) {
    if ((rc = enqueue_step(g, true, 0, nullptr))) return rc;
  } else {
    const int phase = g->desc.rotate_split ? (int)(g->step % g->dim) : 0;
    if ((rc = get_graph(g, phase))) return rc;
    IB_CUDA(cudaGraphLaunch(g->graph[phase], g->s));
  }
  g->step++;
  return IB_OK;
}

// device allocations of one adjoint run, freed together
struct DevPool {
  std::vector<void *> ptrs;
  ~DevPool() {
    for (void *p : ptrs) cudaFree(p);
  }
  char *get(size_t bytes) {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 256) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return (char *)p;
  }
};

inline size_t pad256(size_t b) { return (b + 255) / 256 * 256; }

// Byte sizes of the blocks that make up the state S^n: the fields u, p,
// psi, Nold, div (the first 2d + 3 slots of the field allocation), the
// marker positions X (d nm FP64) and U^{n-1} (d nm of the field precision).
struct StateSizes {
  size_t fbytes, fields, X, Uold;
};

StateSizes state_sizes(const ib_grid_s *g) {
  StateSizes z;
  z.fbytes = pad256((size_t)g->cells * g->esz);
  z.fields = z.fbytes * (2 * g->dim + 3);
  z.X = pad256(sizeof(double) * g->dim * g->nm);
  z.Uold = pad256(g->esz * g->dim * g->nm);
  return z;
}

int copy_state(ib_grid_s *g, char *buf, bool save) {
  const StateSizes z = state_sizes(g);
  char *blk[3] = {(char *)g->fields, (char *)g->X[0], (char *)g->Uold[0]};
  const size_t len[3] = {z.fields, sizeof(double) * g->dim * g->nm, g->esz * g->dim * g->nm};
  const size_t off[3] = {0, z.fields, z.fields + z.X};
  for (int i = 0; i < 3; ++i) {
    if (!len[i]) continue;
    if (save) IB_CUDA(cudaMemcpyAsync(buf + off[i], blk[i], len[i], cudaMemcpyDeviceToDevice, g->s));
    else IB_CUDA(cudaMemcpyAsync(blk[i], buf + off[i], len[i], cudaMemcpyDeviceToDevice, g->s));
  }
  return IB_OK;
}

// After a restore: the grid locations of X are stale (recomputed here).
int relocate(ib_grid_s *g) {
  g->loc_valid = false;
  return ensure_loc(g);
}

template <typename T>
int adjoint_t(ib_grid_s *g, int n_steps, int ck, const double *X_target, double *loss, double *dkappa) {
  const int d = g->dim;
  const int64_t nm = g->nm, ne = g->ne;
  const StateSizes z = state_sizes(g);
  const size_t ck_bytes = z.fields + z.X + z.Uold;
  const size_t tape_fields = z.fbytes * d;  // u^n
  const size_t tape_bytes = tape_fields + z.X + z.Uold;
  const int nseg = (n_steps + ck - 1) / ck;
  const int64_t s0 = g->step;
  DevPool pool;
  char *cks = pool.get(ck_bytes * (nseg + 1));  // segment starts + the final state
  char *tape = pool.get(tape_bytes * (size_t)(n_steps < ck ? (n_steps > 0 ? n_steps : 1) : ck));
  char *adjf = pool.get(z.fbytes * (4 * d + 4));
  const size_t mbytes = pad256(sizeof(double) * d * (nm + 1)), tbytes = pad256(sizeof(T) * d * (nm + 1));
  char *adjm = pool.get(2 * mbytes + 3 * tbytes + pad256(sizeof(double) * (ne + 1)));
  // stencil scratch of the marker adjoint: 2 sets of 3 first nodes and 12
  // weights and derivatives per (marker, component)
  const int64_t npair = nm * d + 1;
  const size_t sbytes = pad256(sizeof(int32_t) * 3 * npair), swbytes = pad256(sizeof(T) * 12 * npair);
  char *adjs = pool.get(2 * (sbytes + 2 * swbytes));
  if (!cks || !tape || !adjf || !adjm || !adjs)
    return fail(IB_ERR_OOM, "adjoint: %zu bytes of checkpoints and tape do not fit",
                ck_bytes * (nseg + 1) + tape_bytes * ck);
  // forward with checkpoints
  for (int sg = 0; sg < nseg; ++sg) {
    int rc = copy_state(g, cks + ck_bytes * sg, true);
    if (rc) return rc;
    const int len = std::min(ck, n_steps - sg * ck);
    for (int j = 0; j < len; ++j)
      if ((rc = forward_one(g))) return rc;
  }
  int rc = copy_state(g, cks + ck_bytes * nseg, true);
  if (rc) return rc;
  // loss and its gradient with respect to the final positions (host, FP64)
  std::vector<double> X(d * nm), Xb(d * nm);
  std::vector<int32_t> perm(nm);
  if (nm) {
    IB_CUDA(cudaMemcpyAsync(X.data(), g->X[0], sizeof(double) * d * nm, cudaMemcpyDeviceToHost, g->s));
    IB_CUDA(cudaMemcpyAsync(perm.data(), g->perm, sizeof(int32_t) * nm, cudaMemcpyDeviceToHost, g->s));
  }
  IB_CUDA(cudaStreamSynchronize(g->s));
  double L = 0.0;
  for (int64_t k = 0; k < nm; ++k)
    for (int a = 0; a < d; ++a) {
      const double r = X[a * nm + k] - X_target[(int64_t)perm[k] * d + a];
      if (!isfinite(r)) return fail(IB_ERR_NONFINITE, "adjoint: non-finite marker position");
      L += r * r;
      Xb[a * nm + k] = 2.0 * r;
    }
  *loss = L;
  // adjoint state
  AdjFields<T> f;
  AdjMarkers<T> am;
  memset(&f, 0, sizeof(f));
  memset(&am, 0, sizeof(am));
  {
    char *b = adjf;
    int slot = 0;
    auto nxt = [&]() { return (T *)(b + z.fbytes * slot++); };
    for (int a = 0; a < d; ++a) f.ub[a] = nxt();
    f.pb = nxt();
    f.psib = nxt();
    for (int a = 0; a < d; ++a) f.nbar[a] = nxt();
    f.divb = nxt();
    f.q = nxt();
    for (int a = 0; a < d; ++a) f.rb[a] = nxt();
    for (int a = 0; a < d; ++a) f.vv[a] = nxt();
    for (int a = d; a < 3; ++a) {
      f.ub[a] = f.ub[d - 1];
      f.nbar[a] = f.nbar[d - 1];
      f.rb[a] = f.rb[d - 1];
      f.vv[a] = f.vv[d - 1];
    }
  }
  f.cells = g->cells;
  f.dim = d;
  for (int a = 0; a < 3; ++a) {
    f.n[a] = g->n[a];
    f.ih[a] = (T)(1.0 / g->h[a]);
  }
  const ib_grid_desc &D = g->desc;
  const bool gm1 = D.scheme == IB_GM1;
  f.chi_mu_half = gm1 ? T(0) : (T)(0.5 * D.chi * D.mu);
  f.p_keep = gm1 ? T(0) : T(1);
  f.psi_w = gm1 ? T(0) : T(1);
  f.rho_dt = (T)(D.rho / D.dt);
  f.dt_mu_rho = (T)(D.dt * D.mu / D.rho);
  f.dt_rho = (T)(D.dt / D.rho);
  f.dt = (T)D.dt;
  double *Xbd = (double *)adjm, *Xhb = (double *)(adjm + mbytes);
  T *Ub = (T *)(adjm + 2 * mbytes), *Uoldb = (T *)(adjm + 2 * mbytes + tbytes), *Gb = (T *)(adjm + 2 * mbytes + 2 * tbytes);
  double *dk = (double *)(adjm + 2 * mbytes + 3 * tbytes);
  IB_CUDA(cudaMemsetAsync(adjf, 0, z.fbytes * (4 * d + 4), g->s));
  IB_CUDA(cudaMemsetAsync(adjm, 0, 2 * mbytes + 3 * tbytes + pad256(sizeof(double) * (ne + 1)), g->s));
  if (nm) IB_CUDA(cudaMemcpyAsync(Xbd, Xb.data(), sizeof(double) * d * nm, cudaMemcpyHostToDevice, g->s));
  for (int a = 0; a < 3; ++a) {
    const int aa = a < d ? a : d - 1;
    am.U[a] = (T *)g->U[aa];
    am.Xh[a] = g->Xh[aa];
    am.G[a] = (T *)g->G[aa];
    am.Gb[a] = Gb + aa * nm;
    am.Xhb[a] = Xhb + aa * nm;
    am.Xb[a] = Xbd + aa * nm;
    am.Ub[a] = Ub + aa * nm;
    am.Uoldb[a] = Uoldb + aa * nm;
    am.inv_h[a] = 1.0 / g->h[a];
    am.n[a] = g->n[a];
  }
  am.row = g->row;
  am.col = g->col;
  am.kap = g->kap;
  am.cedge = g->cedge;
  am.dk = dk;
  am.nm = nm;
  am.dt = D.dt;
  am.H = D.H;
  am.inv_vol = 1.0;
  for (int a = 0; a < d; ++a) am.inv_vol /= g->h[a];
  am.dim = d;
  am.kernel = D.kernel;
  for (int st = 0; st < 2; ++st) {
    char *b = adjs + st * (sbytes + 2 * swbytes);
    am.stb[st] = (int32_t *)b;
    am.stw[st] = (T *)(b + sbytes);
    am.stdw[st] = (T *)(b + sbytes + swbytes);
  }
  SweepArgs<T> sa;
  memset(&sa, 0, sizeof(sa));
  for (int a = 0; a < 3; ++a) {
    sa.n[a] = g->n[a];
    sa.inv_h[a] = (T)(1.0 / g->h[a]);
  }
  sa.dim = d;
  // reverse sweep over the segments
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int len = std::min(ck, n_steps - sg * ck);
    const int64_t s_seg = s0 + (int64_t)sg * ck;
    if ((rc = copy_state(g, cks + ck_bytes * sg, false))) return rc;
    g->step = s_seg;
    if ((rc = relocate(g))) return rc;
    for (int j = 0; j < len; ++j) {  // replay, storing u^n, X^n, U^{n-1}
      char *t = tape + tape_bytes * j;
      IB_CUDA(cudaMemcpyAsync(t, g->fields, tape_fields, cudaMemcpyDeviceToDevice, g->s));
      if (nm) {
        IB_CUDA(cudaMemcpyAsync(t + tape_fields, g->X[0], sizeof(double) * d * nm, cudaMemcpyDeviceToDevice, g->s));
        IB_CUDA(cudaMemcpyAsync(t + tape_fields + z.X, g->Uold[0], g->esz * d * nm, cudaMemcpyDeviceToDevice, g->s));
      }
      if ((rc = forward_one(g))) return rc;
    }
    for (int j = len - 1; j >= 0; --j) {  // adjoint steps, last first
      char *t = tape + tape_bytes * j;
      const int first = s_seg + j == 0;
      const T *u[3];
      for (int a = 0; a < 3; ++a) u[a] = (const T *)(t + z.fbytes * (a < d ? a : d - 1));
      // Steps 3e-3f: q = A^{-1}(psi_bar + p_bar), then the bars of D.u' and u'
      IB_CUDA(adjoint_fields_a<T>(f, g->s));
      sa.f[0] = sa.f[1] = sa.f[2] = f.q;
      for (int ax = 0; ax < d; ++ax) {
        sa.co = chain_coef<T>(g->coef[1], kAxes, ax, d);
        IB_CUDA(launch_sweep<T>(ax, PRO_LOAD, EPI_STORE, 1, sa, g->s, g->tune[ax]));
      }
      IB_CUDA(adjoint_fields_b<T>(f, g->s));
      // Steps 3c-3d: R_bar = M^{-1} u'_bar
      for (int a = 0; a < 3; ++a) sa.f[a] = f.rb[a];
      for (int ax = 0; ax < d; ++ax) {
        sa.co = chain_coef<T>(g->coef[0], kAxes, ax, d);
        IB_CUDA(launch_sweep<T>(ax, PRO_LOAD, EPI_STORE, d, sa, g->s, g->tune[ax]));
      }
      // Steps 3a-3b
      IB_CUDA(adjoint_fields_c<T>(f, u, first, g->s));
      // Steps 1a-2b
      if (nm) {
        for (int a = 0; a < 3; ++a) {
          const int aa = a < d ? a : d - 1;
          am.X[a] = (const double *)(t + tape_fields) + aa * nm;
          am.Uold[a] = (const T *)(t + tape_fields + z.X) + aa * nm;
        }
        am.first = first;
        IB_CUDA(adjoint_markers_pre<T>(am, u, g->s));
        MarkerArgs mf = marker_args(g, first);
        mf.frac_force = 0;  // the stored fractions belong to the forward run, not to X^{n+1/2} here
        IB_CUDA(launch_force<T>(mf, g->s));
        IB_CUDA(cudaMemsetAsync(Xhb, 0, sizeof(double) * d * nm, g->s));
        const T *rbc[3] = {f.rb[0], f.rb[1], f.rb[2]};
        IB_CUDA(adjoint_markers_post<T>(am, rbc, f.dt_rho, u, f.ub, g->s));
      }
    }
  }
  // leave the grid in the final state, as ib_step would
  if ((rc = copy_state(g, cks + ck_bytes * nseg, false))) return rc;
  g->step = s0 + n_steps;
  if ((rc = relocate(g))) return rc;
  if (ne) IB_CUDA(cudaMemcpyAsync(dkappa, dk, sizeof(double) * ne, cudaMemcpyDeviceToHost, g->s));
  IB_CUDA(cudaStreamSynchronize(g->s));
  return IB_OK;
}

bool valid_n(int n) { return n >= 8 && n <= 512; }

// Host view of an input array that may live in host or device memory: device
// (and managed) arrays are copied into tmp on the grid's stream.
template <typename T>
int host_view(ib_grid_s *g, const T *p, int64_t count, std::vector<T> &tmp, const T **out) {
  *out = p;
  if (!p || count <= 0) return IB_OK;
  cudaPointerAttributes at;
  IB_CUDA(cudaPointerGetAttributes(&at, p));
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return IB_OK;
  tmp.resize((size_t)count);
  IB_CUDA(cudaMemcpyAsync(tmp.data(), p, (size_t)count * sizeof(T), cudaMemcpyDeviceToHost, g->s));
  IB_CUDA(cudaStreamSynchronize(g->s));
  *out = tmp.data();
  return IB_OK;
}

}  // namespace

extern "C" {

const char *ib_error_string(int code) {
  switch (code) {
    case IB_OK: return "ok";
    case IB_ERR_ARG: return "invalid argument";
    case IB_ERR_OOM: return "out of memory";
    case IB_ERR_CUDA: return "CUDA error";
    case IB_ERR_NONFINITE: return "non-finite value in the state";
    case IB_ERR_TIMEOUT: return "device wait timed out";
    case IB_ERR_STATE: return "call not allowed in the current state";
    default: return "unknown error";
  }
}

const char *ib_last_error(void) { return g_last_error.c_str(); }

int ib_create_grid(const ib_grid_desc *desc, ib_grid_t *out) {
  if (!desc || !out) return fail(IB_ERR_ARG, "null argument");
  *out = nullptr;
  const ib_grid_desc &D = *desc;
  if (D.dim != 2 && D.dim != 3) return fail(IB_ERR_ARG, "dim must be 2 or 3");
  for (int a = 0; a < D.dim; ++a)
    if (!valid_n(D.n[a])) return fail(IB_ERR_ARG, "n[%d] = %d outside [8, 512]", a, D.n[a]);
  if (!(D.H > 0) || !(D.rho > 0) || !(D.mu >= 0) || !(D.dt > 0) || !(D.chi >= 0))
    return fail(IB_ERR_ARG, "H, rho, dt must be > 0 and mu, chi >= 0");
  if (D.precision != IB_FP32 && D.precision != IB_FP64) return fail(IB_ERR_ARG, "precision");
  if (D.kernel != IB_DELTA_PESKIN4 && D.kernel != IB_DELTA_COS4) return fail(IB_ERR_ARG, "kernel");
  if (D.scheme != IB_GM2 && D.scheme != IB_GM1) return fail(IB_ERR_ARG, "scheme");
  ib_grid_s *g = new ib_grid_s();
  g->desc = D;
  g->dim = D.dim;
  g->prec = D.precision;
  g->esz = D.precision == IB_FP32 ? 4 : 8;
  for (int a = 0; a < D.dim; ++a) {
    g->n[a] = D.n[a];
    g->h[a] = D.H / D.n[a];
  }
  g->cells = (long long)g->n[0] * g->n[1] * g->n[2];
  g->user = (cudaStream_t)D.stream;
  auto cleanup = [&](int rc) {
    ib_destroy_grid(g);
    return rc;
  };
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (cudaStreamCreateWithFlags(&g->s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithPriority(&g->s2, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return cleanup(fail(IB_ERR_CUDA, "stream/event creation failed"));
  const int d = g->dim;
  const int nf = 3 * d + 3;
  const size_t fbytes = ((size_t)g->cells * g->esz + 255) / 256 * 256;
  if (cudaMalloc(&g->fields, fbytes * nf) != cudaSuccess)
    return cleanup(fail(IB_ERR_OOM, "field allocation of %zu bytes failed", fbytes * nf));
  char *b = (char *)g->fields;
  int slot = 0;
  for (int a = 0; a < d; ++a) g->u[a] = b + fbytes * slot++;
  g->p = b + fbytes * slot++;
  g->psi = b + fbytes * slot++;
  for (int a = 0; a < d; ++a) g->Nold[a] = b + fbytes * slot++;
  g->div = b + fbytes * slot++;
  for (int a = 0; a < d; ++a) g->scr[a] = b + fbytes * slot++;
  for (int a = d; a < 3; ++a) {  // unused third component aliases the second
    g->u[a] = g->u[d - 1];
    g->Nold[a] = g->Nold[d - 1];
    g->scr[a] = g->scr[d - 1];
  }
  if (cudaMemsetAsync(g->fields, 0, fbytes * nf, g->s) != cudaSuccess)
    return cleanup(fail(IB_ERR_CUDA, "memset"));
  const double amom = D.mu * D.dt / (2.0 * D.rho);
  for (int a = 0; a < d; ++a) {
    int rc = upload_coef(make_coef(g->n[a], amom / (g->h[a] * g->h[a])), g->coef[0][a], g->s);
    if (rc == IB_OK) rc = upload_coef(make_coef(g->n[a], 1.0 / (g->h[a] * g->h[a])), g->coef[1][a], g->s);
    if (rc != IB_OK) return cleanup(rc);
  }
  if (cudaStreamSynchronize(g->s) != cudaSuccess) return cleanup(fail(IB_ERR_CUDA, "sync"));
  *out = g;
  return IB_OK;
}

int ib_destroy_grid(ib_grid_t g) {
  if (!g) return IB_OK;
  if (g->s) cudaStreamSynchronize(g->s);
  for (int i = 0; i < 3; ++i)
    if (g->graph[i]) cudaGraphExecDestroy(g->graph[i]);
  for (int k = 0; k < 2; ++k)
    for (int a = 0; a < 3; ++a)
      if (g->coef[k][a].mem) cudaFree(g->coef[k][a].mem);
  if (g->fields) cudaFree(g->fields);
  if (g->mk) cudaFree(g->mk);
  if (g->ev_in) cudaEventDestroy(g->ev_in);
  if (g->ev_out) cudaEventDestroy(g->ev_out);
  if (g->ev_fork) cudaEventDestroy(g->ev_fork);
  if (g->ev_join) cudaEventDestroy(g->ev_join);
  if (g->s2) cudaStreamDestroy(g->s2);
  if (g->s) cudaStreamDestroy(g->s);
  delete g;
  return IB_OK;
}

int ib_add_fiber(ib_grid_t g, const double *X0_in, int64_t n_markers, const int32_t *edges_in,
                 const double *kappa_in, const double *rest_in, int64_t n_edges, const int32_t *tris_in,
                 int64_t n_tris, int32_t *fiber_id_out) {
  if (!g) return fail(IB_ERR_ARG, "null grid");
  if (g->step != 0 || g->markers_uploaded) return fail(IB_ERR_STATE, "fibers can only be added before the first step");
  if (n_markers < 0 || n_edges < 0 || n_tris < 0) return fail(IB_ERR_ARG, "negative count");
  if (n_markers > 0 && !X0_in) return fail(IB_ERR_ARG, "null X0");
  if (n_edges > 0 && (!edges_in || !kappa_in)) return fail(IB_ERR_ARG, "null edges or kappa");
  if (g->nm + n_markers > ((int64_t)1 << 25)) return fail(IB_ERR_ARG, "more than 2^25 markers");
  const int d = g->dim;
  // every array may be host or device memory
  std::vector<double> tX, tK, tR;
  std::vector<int32_t> tE, tT;
  const double *X0, *kappa, *rest_len;
  const int32_t *edges, *tris;
  int rc = enter(g);
  if (rc) return rc;
  if ((rc = host_view(g, X0_in, n_markers * d, tX, &X0)) || (rc = host_view(g, edges_in, 2 * n_edges, tE, &edges)) ||
      (rc = host_view(g, kappa_in, n_edges, tK, &kappa)) || (rc = host_view(g, rest_in, n_edges, tR, &rest_len)) ||
      (rc = host_view(g, tris_in, d == 3 ? 3 * n_tris : 0, tT, &tris)))
    return rc;
  if ((rc = leave(g))) return rc;
  for (int64_t i = 0; i < n_markers * d; ++i)
    if (!isfinite(X0[i])) return fail(IB_ERR_NONFINITE, "non-finite marker position");
  for (int64_t e = 0; e < 2 * n_edges; ++e)
    if (edges[e] < 0 || edges[e] >= n_markers) return fail(IB_ERR_ARG, "edge index %d out of range", edges[e]);
  if (d == 3)
    for (int64_t t = 0; t < 3 * n_tris; ++t)
      if (!tris || tris[t] < 0 || tris[t] >= n_markers) return fail(IB_ERR_ARG, "triangle index out of range");
  const int32_t off = (int32_t)g->nm;
  g->hX.insert(g->hX.end(), X0, X0 + n_markers * d);
  for (int64_t e = 0; e < n_edges; ++e) {
    g->hE.push_back(edges[2 * e] + off);
    g->hE.push_back(edges[2 * e + 1] + off);
    g->hK.push_back(kappa[e]);
    g->hR.push_back(rest_len ? rest_len[e] : 0.0);
  }
  if (d == 3)
    for (int64_t t = 0; t < 3 * n_tris; ++t) g->hT.push_back(tris[t] + off);
  g->nm += n_markers;
  g->ne += n_edges;
  if (d == 3) g->nt += n_tris;
  if (fiber_id_out) *fiber_id_out = g->nfibers;
  g->nfibers++;
  return IB_OK;
}

int ib_set_velocity(ib_grid_t g, int comp, const void *src, int on_device) {
  if (!g || !src) return fail(IB_ERR_ARG, "null argument");
  if (comp < 0 || comp >= g->dim) return fail(IB_ERR_ARG, "component %d", comp);
  if (g->step != 0) return fail(IB_ERR_STATE, "velocity can only be set before the first step");
  int rc = enter(g);
  if (rc) return rc;
  IB_CUDA(cudaMemcpyAsync(g->u[comp], src, g->cells * g->esz,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->s));
  if (!on_device) IB_CUDA(cudaStreamSynchronize(g->s));
  g->div_valid = false;
  return leave(g);
}

int ib_step(ib_grid_t g, int n_steps) {
  if (!g) return fail(IB_ERR_ARG, "null grid");
  if (n_steps < 0) return fail(IB_ERR_ARG, "n_steps < 0");
  if (n_steps == 0) return IB_OK;
  int rc = enter(g);
  if (rc) return rc;
  if ((rc = prepare(g))) return rc;
  for (int i = 0; i < n_steps; ++i) {
    if (g->resort_every > 0 && g->step > 0 && g->step % g->resort_every == 0 && (rc = resort_markers(g))) return rc;
    if (g->step == 0) {
      if ((rc = enqueue_step(g, true, 0, nullptr))) return rc;
    } else {
      const int phase = g->desc.rotate_split ? (int)(g->step % g->dim) : 0;
      if ((rc = get_graph(g, phase))) return rc;
      IB_CUDA(cudaGraphLaunch(g->graph[phase], g->s));
    }
    g->step++;
  }
  return leave(g);
}

int ib_profile_step(ib_grid_t g, int n_steps, float *kernel_ms, int max_kernels, int *n_kernels) {
  if (!g || !kernel_ms || n_steps < 0) return fail(IB_ERR_ARG, "bad argument");
  const int nslots = 12;  // marks 0..11 (see below) + one end mark
  const int nk = 11;      // interp, update, force, spread, rhs, 3 momentum + 3 psi sweeps
  cudaEvent_t ev[nslots + 1];
  for (int i = 0; i <= nslots; ++i) IB_CUDA(cudaEventCreate(&ev[i]));
  std::vector<double> tot(nk, 0.0);
  int rc = enter(g);
  if (!rc) rc = prepare(g);
  for (int i = 0; i < n_steps && !rc; ++i) {
    const int phase = g->desc.rotate_split ? (int)(g->step % g->dim) : 0;
    for (int k = 0; k <= nslots; ++k) cudaEventRecord(ev[k], g->s);
    rc = enqueue_step(g, g->step == 0, phase, ev);
    if (rc) break;
    cudaEventRecord(ev[nslots], g->s);
    if (cudaEventSynchronize(ev[nslots]) != cudaSuccess) {
      rc = fail(IB_ERR_CUDA, "profiling sync");
      break;
    }
    // marks: 0 before interp, 1 after interp, 2 after update, 3 after force,
    // 4 after rhs, 5 after spread, 6 + s after the s-th momentum sweep, 9 + s
    // after the s-th psi sweep (s in split order)
    float ms;
    const int span[5][2] = {{0, 1}, {1, 2}, {2, 3}, {4, 5}, {3, 4}};  // interp, update, force, spread, rhs
    for (int k = 0; k < 5; ++k) {
      cudaEventElapsedTime(&ms, ev[span[k][0]], ev[span[k][1]]);
      tot[k] += ms;
    }
    for (int q = 0; q < g->dim; ++q) {
      cudaEventElapsedTime(&ms, ev[5 + q], ev[6 + q]);
      tot[5 + q] += ms;
    }
    for (int q = 0; q < g->dim; ++q) {
      cudaEventElapsedTime(&ms, q == 0 ? ev[6 + g->dim - 1] : ev[8 + q], ev[9 + q]);
      tot[8 + q] += ms;
    }
    g->step++;
  }
  for (int i = 0; i <= nslots; ++i) cudaEventDestroy(ev[i]);
  if (rc) return rc;
  for (int k = 0; k < nk && k < max_kernels; ++k) kernel_ms[k] = (float)tot[k];
  if (n_kernels) *n_kernels = nk < max_kernels ? nk : max_kernels;
  return leave(g);
}

int ib_sweep_config(ib_grid_t g, int axis, int *cfg) {
  if (!g || !cfg || axis < 0 || axis >= g->dim) return fail(IB_ERR_ARG, "bad argument");
  int rc = enter(g);
  if (!rc) rc = prepare(g);
  if (!rc) rc = leave(g);
  if (rc) return rc;
  const int id = g->tune[axis];
  sweep_config_shape(axis, id, g->n[axis], &cfg[1], &cfg[2], &cfg[3]);
  cfg[0] = id;
  return IB_OK;
}

int ib_fix_sweep_config(ib_grid_t g, int axis, int id) {
  if (!g || axis < 0 || axis >= g->dim) return fail(IB_ERR_ARG, "bad argument");
  if (g->tuned || g->step != 0) return fail(IB_ERR_STATE, "sweep configurations are fixed before the first step");
  int cand[24];
  const int nc = sweep_candidates(axis, g->n[axis], g->n[0], g->prec == IB_FP64, cand, 24);
  bool ok = false;
  for (int i = 0; i < nc; ++i) ok = ok || cand[i] == id;
  if (!ok) return fail(IB_ERR_ARG, "configuration %d is not a candidate for axis %d of this grid", id, axis);
  g->tune[axis] = g->tune_psi[axis] = id;
  g->tune_r[axis] = g->tune_div[axis] = g->tune_addu[axis] = g->tune_p[axis] = id == kTmaCfg ? -1 : id;
  g->fixed[axis] = true;
  return IB_OK;
}

int ib_resort_markers(ib_grid_t g) {
  if (!g) return fail(IB_ERR_ARG, "null grid");
  int rc = enter(g);
  if (!rc) rc = upload_markers(g);
  if (!rc) rc = resort_markers(g);
  if (rc) return rc;
  return leave(g);
}

int ib_set_resort_interval(ib_grid_t g, int every) {
  if (!g || every < 0) return fail(IB_ERR_ARG, "bad argument");
  g->resort_every = every;
  return IB_OK;
}

const char *ib_kernel_name(int slot) {
  // sweeps are numbered by their position in the step's split order
  static const char *names[] = {"interp",      "update",      "force",       "spread",
                                "rhs",         "mom_sweep_1", "mom_sweep_2", "mom_sweep_3",
                                "psi_sweep_1", "psi_sweep_2", "psi_sweep_3"};
  return (slot >= 0 && slot < 11) ? names[slot] : "";
}

int ib_read_fields(ib_grid_t g, unsigned field_mask, void *dst, size_t bytes, int dst_on_device) {
  if (!g || !dst) return fail(IB_ERR_ARG, "null argument");
  void *src[6] = {g->u[0], g->u[1], g->dim == 3 ? g->u[2] : nullptr, g->p, g->psi, g->div};
  size_t need = 0;
  for (int b = 0; b < 6; ++b)
    if (field_mask & (1u << b)) {
      if (!src[b]) return fail(IB_ERR_ARG, "field bit %d not present in %dD", b, g->dim);
      need += g->cells * g->esz;
    }
  if (need != bytes) return fail(IB_ERR_ARG, "bytes = %zu, fields need %zu", bytes, need);
  int rc = enter(g);
  if (rc) return rc;
  if ((field_mask & IB_FIELD_DIV) && (rc = ensure_div(g))) return rc;
  char *o = (char *)dst;
  for (int b = 0; b < 6; ++b)
    if (field_mask & (1u << b)) {
      IB_CUDA(cudaMemcpyAsync(o, src[b], g->cells * g->esz,
                              dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->s));
      o += g->cells * g->esz;
    }
  if (!dst_on_device) IB_CUDA(cudaStreamSynchronize(g->s));
  return leave(g);
}

int ib_read_markers(ib_grid_t g, double *X, int64_t n, int dst_on_device) {
  if (!g || (!X && n)) return fail(IB_ERR_ARG, "null argument");
  if (n != g->nm) return fail(IB_ERR_ARG, "n = %lld, grid has %lld markers", (long long)n, (long long)g->nm);
  if (n == 0) return IB_OK;
  int rc = enter(g);
  if (rc) return rc;
  if ((rc = upload_markers(g))) return rc;
  const int d = g->dim;
  // SoA on the device -> [n][dim] staging -> caller
  IB_CUDA(launch_markers_layout(g->stage, g->X, g->perm, n, d, 0, g->s));
  IB_CUDA(cudaMemcpyAsync(X, g->stage, sizeof(double) * n * d,
                          dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->s));
  if (!dst_on_device) IB_CUDA(cudaStreamSynchronize(g->s));
  return leave(g);
}

int ib_set_markers(ib_grid_t g, const double *X, int64_t n, int src_on_device) {
  if (!g || (!X && n)) return fail(IB_ERR_ARG, "null argument");
  if (n != g->nm) return fail(IB_ERR_ARG, "n = %lld, grid has %lld markers", (long long)n, (long long)g->nm);
  if (n == 0) return IB_OK;
  int rc = enter(g);
  if (rc) return rc;
  if ((rc = upload_markers(g))) return rc;
  const int d = g->dim;
  IB_CUDA(cudaMemcpyAsync(g->stage, X, sizeof(double) * n * d,
                          src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->s));
  IB_CUDA(launch_markers_layout(g->stage, g->X, g->perm, n, d, 1, g->s));
  g->loc_valid = false;
  if ((rc = ensure_loc(g))) return rc;
  if (!src_on_device) IB_CUDA(cudaStreamSynchronize(g->s));
  return leave(g);
}

int ib_diagnostics(ib_grid_t g, ib_diag *out) {
  if (!g || !out) return fail(IB_ERR_ARG, "null argument");
  int rc = enter(g);
  if (!rc) rc = prepare(g);
  if (rc) return rc;
  IB_CUDA(cudaMemsetAsync(g->acc, 0, 8 * sizeof(double), g->s));
  if (g->prec == IB_FP32) {
    const float *uc[3] = {(const float *)g->u[0], (const float *)g->u[1], (const float *)g->u[2]};
    IB_CUDA(launch_field_diag<float>(g->dim, uc, (const float *)g->p, (const float *)g->div, g->n, g->acc, g->s));
  } else {
    const double *uc[3] = {(const double *)g->u[0], (const double *)g->u[1], (const double *)g->u[2]};
    IB_CUDA(launch_field_diag<double>(g->dim, uc, (const double *)g->p, (const double *)g->div, g->n, g->acc,
                                      g->s));
  }
  const double *Xc[3] = {g->X[0], g->X[1], g->X[2]};
  IB_CUDA(launch_marker_diag(g->dim, Xc, g->nm, g->edges, g->ekap, g->erest, g->ne, g->tris, g->nt, g->desc.H,
                             g->acc, g->s));
  double acc[8];
  IB_CUDA(cudaMemcpyAsync(acc, g->acc, sizeof(acc), cudaMemcpyDeviceToHost, g->s));
  IB_CUDA(cudaStreamSynchronize(g->s));
  double vol = 1.0;
  for (int a = 0; a < g->dim; ++a) vol *= g->h[a];
  out->div_l2 = sqrt(vol * acc[0]);
  out->div_max = acc[1];
  out->kinetic = 0.5 * g->desc.rho * vol * acc[2];
  out->volume = acc[3];
  out->elastic = acc[4];
  out->step = g->step;
  if ((rc = leave(g))) return rc;
  if (take_wait_timeout()) return fail(IB_ERR_TIMEOUT, "a bounded device wait ran out in an earlier launch");
  if (acc[5] != 0.0 || !isfinite(acc[0]) || !isfinite(acc[2]) || !isfinite(acc[3]))
    return fail(IB_ERR_NONFINITE, "%g non-finite values in the state", acc[5]);
  return IB_OK;
}

int ib_cyclic_solve_lines(int precision, int dim, const int n[3], int axis, double r, const void *in, void *out,
                          void *stream) {
  if (!n || !in || !out) return fail(IB_ERR_ARG, "null argument");
  if ((dim != 2 && dim != 3) || axis < 0 || axis >= dim) return fail(IB_ERR_ARG, "dim/axis");
  if (precision != IB_FP32 && precision != IB_FP64) return fail(IB_ERR_ARG, "precision");
  if (!(r >= 0)) return fail(IB_ERR_ARG, "r must be >= 0");
  for (int a = 0; a < dim; ++a)
    if (!valid_n(n[a])) return fail(IB_ERR_ARG, "n[%d] = %d outside [8, 512]", a, n[a]);
  cudaStream_t s = (cudaStream_t)stream;
  DevCoef *c;
  int rc = cached_coef(n[axis], r, s, &c);
  if (rc) return rc;
  if (precision == IB_FP32) {
    SweepArgs<float> a;
    memset(&a, 0, sizeof(a));
    a.f[0] = (float *)out;
    a.fin[0] = (const float *)in;
    for (int q = 0; q < 3; ++q) a.n[q] = q < dim ? n[q] : 1;
    a.dim = dim;
    a.co = c->f;
    IB_CUDA(launch_sweep<float>(axis, PRO_LOAD, EPI_STORE, 1, a, s));
  } else {
    SweepArgs<double> a;
    memset(&a, 0, sizeof(a));
    a.f[0] = (double *)out;
    a.fin[0] = (const double *)in;
    for (int q = 0; q < 3; ++q) a.n[q] = q < dim ? n[q] : 1;
    a.dim = dim;
    a.co = c->d;
    IB_CUDA(launch_sweep<double>(axis, PRO_LOAD, EPI_STORE, 1, a, s));
  }
  return IB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Checkpoint / resume: the state S^n as a host byte image.
//   header | fields u[d], p, psi, Nold[d], div (n0 n1 n2 elements each, field
//   precision, grid order) | X [nm][d] FP64 | U^{n-1} [nm][d] field precision
//   (markers in the caller's order)

namespace {

struct StateHeader {
  char magic[8];  // "IBGMSTAT"
  int32_t version, dim, n[3], precision, scheme;
  int64_t nm, ne, step;
};
static_assert(sizeof(StateHeader) == 64, "the state image header is 64 bytes");

// the field part of the image: u[0..d), p, psi, Nold[0..d), div
int state_fields(ib_grid_s *g, void *out[9]) {
  int k = 0;
  for (int a = 0; a < g->dim; ++a) out[k++] = g->u[a];
  out[k++] = g->p;
  out[k++] = g->psi;
  for (int a = 0; a < g->dim; ++a) out[k++] = g->Nold[a];
  out[k++] = g->div;
  return k;
}

size_t state_bytes(const ib_grid_s *g) {
  return sizeof(StateHeader) + g->esz * (size_t)g->cells * (2 * g->dim + 3) +
         (sizeof(double) + g->esz) * (size_t)g->nm * g->dim;
}

}  // namespace

extern "C" {

int ib_state_size(ib_grid_t g, size_t *bytes) {
  if (!g || !bytes) return fail(IB_ERR_ARG, "null argument");
  *bytes = state_bytes(g);
  return IB_OK;
}

int ib_save_state(ib_grid_t g, void *dst, size_t bytes) {
  if (!g || !dst) return fail(IB_ERR_ARG, "null argument");
  if (bytes != state_bytes(g)) return fail(IB_ERR_ARG, "bytes = %zu, the state needs %zu", bytes, state_bytes(g));
  int rc = enter(g);
  if (!rc) rc = prepare(g);
  if (rc) return rc;
  const int d = g->dim;
  const int64_t nm = g->nm;
  StateHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, "IBGMSTAT", 8);
  h.version = 1;
  h.dim = d;
  for (int a = 0; a < 3; ++a) h.n[a] = g->n[a];
  h.precision = g->prec;
  h.scheme = g->desc.scheme;
  h.nm = nm;
  h.ne = g->ne;
  h.step = g->step;
  char *o = (char *)dst;
  memcpy(o, &h, sizeof(h));
  o += sizeof(h);
  const size_t fb = g->esz * (size_t)g->cells;
  void *fields[9];
  const int nf = state_fields(g, fields);
  for (int i = 0; i < nf; ++i) {
    IB_CUDA(cudaMemcpyAsync(o, fields[i], fb, cudaMemcpyDeviceToHost, g->s));
    o += fb;
  }
  if (nm) {
    IB_CUDA(launch_markers_layout(g->stage, g->X, g->perm, nm, d, 0, g->s));
    IB_CUDA(cudaMemcpyAsync(o, g->stage, sizeof(double) * nm * d, cudaMemcpyDeviceToHost, g->s));
    o += sizeof(double) * nm * d;
    std::vector<char> uold(g->esz * nm * d);
    std::vector<int32_t> perm(nm);
    IB_CUDA(cudaMemcpyAsync(uold.data(), g->Uold[0], uold.size(), cudaMemcpyDeviceToHost, g->s));
    IB_CUDA(cudaMemcpyAsync(perm.data(), g->perm, sizeof(int32_t) * nm, cudaMemcpyDeviceToHost, g->s));
    IB_CUDA(cudaStreamSynchronize(g->s));
    for (int64_t k = 0; k < nm; ++k)
      for (int a = 0; a < d; ++a)
        memcpy(o + g->esz * ((int64_t)perm[k] * d + a), uold.data() + g->esz * (a * nm + k), g->esz);
  }
  IB_CUDA(cudaStreamSynchronize(g->s));
  return leave(g);
}

int ib_load_state(ib_grid_t g, const void *src, size_t bytes) {
  if (!g || !src) return fail(IB_ERR_ARG, "null argument");
  if (bytes != state_bytes(g)) return fail(IB_ERR_ARG, "bytes = %zu, the state needs %zu", bytes, state_bytes(g));
  StateHeader h;
  memcpy(&h, src, sizeof(h));
  if (memcmp(h.magic, "IBGMSTAT", 8) != 0 || h.version != 1) return fail(IB_ERR_ARG, "not a saved state");
  if (h.dim != g->dim || h.n[0] != g->n[0] || h.n[1] != g->n[1] || h.n[2] != g->n[2] || h.precision != g->prec ||
      h.nm != g->nm || h.ne != g->ne || h.scheme != g->desc.scheme || h.step < 0)
    return fail(IB_ERR_ARG, "the saved state belongs to a grid of another shape, precision, scheme or structure");
  int rc = enter(g);
  if (!rc) rc = prepare(g);
  if (rc) return rc;
  const int d = g->dim;
  const int64_t nm = g->nm;
  const char *o = (const char *)src + sizeof(h);
  const size_t fb = g->esz * (size_t)g->cells;
  void *fields[9];
  const int nf = state_fields(g, fields);
  for (int i = 0; i < nf; ++i) {
    IB_CUDA(cudaMemcpyAsync(fields[i], o, fb, cudaMemcpyHostToDevice, g->s));
    o += fb;
  }
  std::vector<char> uold;
  if (nm) {
    IB_CUDA(cudaMemcpyAsync(g->stage, o, sizeof(double) * nm * d, cudaMemcpyHostToDevice, g->s));
    IB_CUDA(launch_markers_layout(g->stage, g->X, g->perm, nm, d, 1, g->s));
    o += sizeof(double) * nm * d;
    std::vector<int32_t> perm(nm);
    IB_CUDA(cudaMemcpyAsync(perm.data(), g->perm, sizeof(int32_t) * nm, cudaMemcpyDeviceToHost, g->s));
    IB_CUDA(cudaStreamSynchronize(g->s));
    uold.resize(g->esz * nm * d);
    for (int64_t k = 0; k < nm; ++k)
      for (int a = 0; a < d; ++a)
        memcpy(uold.data() + g->esz * (a * nm + k), o + g->esz * ((int64_t)perm[k] * d + a), g->esz);
    IB_CUDA(cudaMemcpyAsync(g->Uold[0], uold.data(), uold.size(), cudaMemcpyHostToDevice, g->s));
  }
  g->step = h.step;
  g->div_valid = true;
  g->loc_valid = false;
  if ((rc = ensure_loc(g))) return rc;
  IB_CUDA(cudaStreamSynchronize(g->s));
  return leave(g);
}

}  // extern "C"

extern "C" {

int ib_selftest_wait_timeout(void *stream, int *timed_out) {
  if (!timed_out) return fail(IB_ERR_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  take_wait_timeout();  // start from a clear flag
  IB_CUDA(launch_wait_selftest(1000000ull, s));  // 1 ms
  IB_CUDA(cudaStreamSynchronize(s));
  *timed_out = take_wait_timeout();
  return IB_OK;
}

int ib_split_solve(int precision, int dim, const int n[3], const double r[3], const void *f, void *psi,
                   void *stream) {
  if (!r) return fail(IB_ERR_ARG, "null r");
  for (int a = 0; a < (dim == 3 ? 3 : 2); ++a) {
    int rc = ib_cyclic_solve_lines(precision, dim, n, a, r[a], a == 0 ? f : psi, psi, stream);
    if (rc) return rc;
  }
  return IB_OK;
}

int ib_adjoint_run(ib_grid_t g, int n_steps, int checkpoint_every, const double *X_target, double *loss,
                   double *dkappa) {
  if (!g || !loss || n_steps < 0 || checkpoint_every < 1) return fail(IB_ERR_ARG, "bad argument");
  if (g->nm && !X_target) return fail(IB_ERR_ARG, "null X_target");
  if (g->ne && !dkappa) return fail(IB_ERR_ARG, "null dkappa");
  for (double r : g->hR)
    if (r != 0.0) return fail(IB_ERR_ARG, "the adjoint needs every rest length to be 0");
  int rc = enter(g);
  if (rc) return rc;
  if ((rc = prepare(g))) return rc;
  rc = g->prec == IB_FP32 ? adjoint_t<float>(g, n_steps, checkpoint_every, X_target, loss, dkappa)
                          : adjoint_t<double>(g, n_steps, checkpoint_every, X_target, loss, dkappa);
  if (rc) return rc;
  return leave(g);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// ensembles

// Members are grouped into size classes (same precision, dim and n): within
// a class every kernel of the step has the same template instance and
// launch shape, so each kernel slot of a step is ONE batched launch that
// walks the class's member table (launch_batch); the classes run side by
// side on their own streams, and in each class the marker chain runs beside
// the right-hand side as in a single grid's step.
constexpr size_t kEnsembleGroup = 4;  // members per group of a size class (one batched launch)

struct ib_ensemble_s {
  std::vector<ib_grid_s *> m;
  cudaStream_t s = nullptr, user = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;  // per member: ordering against its own stream
  std::vector<std::vector<int>> cls;  // member indices of each size class
  std::vector<cudaStream_t> cs, cs2;  // per class: main and marker-chain streams
  std::vector<cudaEvent_t> cev_fork, cev_mk, cev_join;
  cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
  int dim = 0;
};

namespace {

// one step of the members of size class c, in batched launches
template <typename T>
int ens_class_step(ib_ensemble_s *e, int c, bool first, int phase) {
  const std::vector<int> &mem = e->cls[c];
  const int n = (int)mem.size();
  std::vector<StepPlan<T>> P(n);
  std::vector<MarkerFieldArgs> mi(n), msp(n);
  std::vector<MarkerArgs> mm(n);
  std::vector<RhsArgs<T>> ra(n);
  std::vector<SweepArgs<T>> sw(n);
  bool markers = false;
  for (int i = 0; i < n; ++i) {
    plan_step<T>(e->m[mem[i]], first, phase, P[i]);
    mm[i] = P[i].m;
    mi[i].m = msp[i].m = P[i].m;
    for (int a = 0; a < 3; ++a) {
      mi[i].f[a] = (void *)P[i].uc[a];
      msp[i].f[a] = (void *)P[i].sc[a];
    }
    ra[i] = P[i].ra;
    markers = markers || P[i].m.nm > 0;
  }
  cudaStream_t s1 = e->cs[c], s2 = e->cs2[c];
  if (markers) {
    IB_CUDA(cudaEventRecord(e->cev_fork[c], s1));
    IB_CUDA(cudaStreamWaitEvent(s2, e->cev_fork[c], 0));
    IB_CUDA(launch_interp_batch<T>(mi.data(), n, s2));
    IB_CUDA(launch_update_batch<T>(mm.data(), n, s2));
    IB_CUDA(launch_force_batch<T>(mm.data(), n, s2));
    IB_CUDA(cudaEventRecord(e->cev_mk[c], s2));
  }
  IB_CUDA(launch_rhs_batch<T>(e->dim, ra.data(), n, s1));
  if (markers) {
    IB_CUDA(cudaStreamWaitEvent(s1, e->cev_mk[c], 0));
    IB_CUDA(launch_spread_batch<T>(msp.data(), n, s1));
  }
  for (int k = 0; k < P[0].nsw; ++k) {
    for (int i = 0; i < n; ++i) sw[i] = P[i].sw[k];
    IB_CUDA(launch_sweep_batch<T>(P[0].ax[k], P[0].pro[k], P[0].epi[k], P[0].nf[k], sw.data(), n, s1,
                                  P[0].cfg_r[k]));
  }
  return IB_OK;
}

// one step of every member: fork from the ensemble stream into the class
// streams, then join back
int ens_enqueue(ib_ensemble_s *e, bool first, int phase) {
  IB_CUDA(cudaEventRecord(e->ev_fork, e->s));
  for (size_t c = 0; c < e->cls.size(); ++c) {
    IB_CUDA(cudaStreamWaitEvent(e->cs[c], e->ev_fork, 0));
    const int rc = e->m[e->cls[c][0]]->prec == IB_FP32 ? ens_class_step<float>(e, (int)c, first, phase)
                                                       : ens_class_step<double>(e, (int)c, first, phase);
    if (rc) return rc;
    IB_CUDA(cudaEventRecord(e->cev_join[c], e->cs[c]));
    IB_CUDA(cudaStreamWaitEvent(e->s, e->cev_join[c], 0));
  }
  return IB_OK;
}

int ens_graph(ib_ensemble_s *e, int phase) {
  if (e->graph[phase]) return IB_OK;
  cudaGraph_t graph;
  IB_CUDA(cudaStreamBeginCapture(e->s, cudaStreamCaptureModeThreadLocal));
  int rc = ens_enqueue(e, false, phase);
  cudaError_t err = cudaStreamEndCapture(e->s, &graph);
  if (rc != IB_OK) {
    if (err == cudaSuccess) cudaGraphDestroy(graph);
    return rc;
  }
  if (err != cudaSuccess) return fail(IB_ERR_CUDA, "ensemble capture: %s", cudaGetErrorString(err));
  err = cudaGraphInstantiate(&e->graph[phase], graph, 0);
  cudaGraphDestroy(graph);
  if (err != cudaSuccess) return fail(IB_ERR_CUDA, "ensemble instantiate: %s", cudaGetErrorString(err));
  return IB_OK;
}

}  // namespace

extern "C" {

int ib_destroy_ensemble(ib_ensemble_t e) {
  if (!e) return IB_OK;
  if (e->s) cudaStreamSynchronize(e->s);
  for (int i = 0; i < 3; ++i)
    if (e->graph[i]) cudaGraphExecDestroy(e->graph[i]);
  for (cudaEvent_t ev : e->ev_join)
    if (ev) cudaEventDestroy(ev);
  for (auto *v : {&e->cev_fork, &e->cev_mk, &e->cev_join})
    for (cudaEvent_t ev : *v)
      if (ev) cudaEventDestroy(ev);
  for (auto *v : {&e->cs, &e->cs2})
    for (cudaStream_t st : *v)
      if (st) cudaStreamDestroy(st);
  if (e->ev_in) cudaEventDestroy(e->ev_in);
  if (e->ev_out) cudaEventDestroy(e->ev_out);
  if (e->ev_fork) cudaEventDestroy(e->ev_fork);
  if (e->s) cudaStreamDestroy(e->s);
  delete e;
  return IB_OK;
}

int ib_create_ensemble(const ib_grid_t *members, int n_members, void *stream, ib_ensemble_t *out) {
  if (!members || !out || n_members < 1) return fail(IB_ERR_ARG, "need at least one member");
  *out = nullptr;
  const ib_grid_s *g0 = members[0];
  if (!g0) return fail(IB_ERR_ARG, "null member");
  for (int i = 0; i < n_members; ++i) {
    const ib_grid_s *g = members[i];
    if (!g) return fail(IB_ERR_ARG, "null member %d", i);
    if (g->dim != g0->dim || g->desc.rotate_split != g0->desc.rotate_split || g->step != g0->step)
      return fail(IB_ERR_STATE, "member %d differs in dim, rotate_split or step count", i);
    for (int j = 0; j < i; ++j)
      if (members[j] == g) return fail(IB_ERR_ARG, "member %d repeated", i);
  }
  ib_ensemble_s *e = new ib_ensemble_s();
  e->dim = g0->dim;
  e->user = (cudaStream_t)stream;
  e->m.assign(members, members + n_members);
  e->ev_join.assign(n_members, nullptr);
  if (cudaStreamCreateWithFlags(&e->s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&e->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&e->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
    ib_destroy_ensemble(e);
    return fail(IB_ERR_CUDA, "ensemble stream/event creation failed");
  }
  for (int i = 0; i < n_members; ++i)
    if (cudaEventCreateWithFlags(&e->ev_join[i], cudaEventDisableTiming) != cudaSuccess) {
      ib_destroy_ensemble(e);
      return fail(IB_ERR_CUDA, "ensemble event creation failed");
    }
  // size classes in order of first appearance, each split into groups of at
  // most kEnsembleGroup members (groups run on their own streams, so the
  // marker stages of some overlap the field stages of others)
  std::vector<std::vector<int>> cls;
  for (int i = 0; i < n_members; ++i) {
    const ib_grid_s *g = members[i];
    size_t c = 0;
    for (; c < cls.size(); ++c) {
      const ib_grid_s *h = members[cls[c][0]];
      if (h->prec == g->prec && h->n[0] == g->n[0] && h->n[1] == g->n[1] && h->n[2] == g->n[2]) break;
    }
    if (c == cls.size()) cls.emplace_back();
    cls[c].push_back(i);
  }
  for (const std::vector<int> &c : cls) {
    const size_t ng = (c.size() + kEnsembleGroup - 1) / kEnsembleGroup;
    for (size_t q = 0; q < ng; ++q) {
      e->cls.emplace_back();
      for (size_t i = q; i < c.size(); i += ng) e->cls.back().push_back(c[i]);
    }
  }
  const size_t nc = e->cls.size();
  e->cs.assign(nc, nullptr);
  e->cs2.assign(nc, nullptr);
  e->cev_fork.assign(nc, nullptr);
  e->cev_mk.assign(nc, nullptr);
  e->cev_join.assign(nc, nullptr);
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  for (size_t c = 0; c < nc; ++c)
    if (cudaStreamCreateWithFlags(&e->cs[c], cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithPriority(&e->cs2[c], cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->cev_fork[c], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->cev_mk[c], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->cev_join[c], cudaEventDisableTiming) != cudaSuccess) {
      ib_destroy_ensemble(e);
      return fail(IB_ERR_CUDA, "ensemble stream/event creation failed");
    }
  for (ib_grid_s *g : e->m) {
    int rc = enter(g);
    if (!rc) rc = prepare(g);
    if (!rc) rc = leave(g);
    if (rc) {
      ib_destroy_ensemble(e);
      return rc;
    }
  }
  *out = e;
  return IB_OK;
}

int ib_ensemble_step(ib_ensemble_t e, int n_steps) {
  if (!e) return fail(IB_ERR_ARG, "null ensemble");
  if (n_steps < 0) return fail(IB_ERR_ARG, "n_steps < 0");
  if (n_steps == 0) return IB_OK;
  for (ib_grid_s *g : e->m)
    if (g->step != e->m[0]->step) return fail(IB_ERR_STATE, "members were stepped separately");
  // order after the caller's stream and after earlier work on every member
  IB_CUDA(cudaEventRecord(e->ev_in, e->user));
  IB_CUDA(cudaStreamWaitEvent(e->s, e->ev_in, 0));
  for (size_t i = 0; i < e->m.size(); ++i) {
    IB_CUDA(cudaEventRecord(e->ev_join[i], e->m[i]->s));
    IB_CUDA(cudaStreamWaitEvent(e->s, e->ev_join[i], 0));
  }
  // capture every phase's graph up front, so that no capture happens between steps
  const int phases = e->m[0]->desc.rotate_split ? e->dim : 1;
  for (int ph = 0; ph < phases; ++ph) {
    int rc = ens_graph(e, ph);
    if (rc) return rc;
  }
  for (int i = 0; i < n_steps; ++i) {
    const int64_t step = e->m[0]->step;
    if (step == 0) {
      int rc = ens_enqueue(e, true, 0);
      if (rc) return rc;
    } else {
      const int phase = e->m[0]->desc.rotate_split ? (int)(step % e->dim) : 0;
      IB_CUDA(cudaGraphLaunch(e->graph[phase], e->s));
    }
    for (ib_grid_s *g : e->m) g->step++;
  }
  // later work on the caller's stream and on every member comes after this
  IB_CUDA(cudaEventRecord(e->ev_out, e->s));
  IB_CUDA(cudaStreamWaitEvent(e->user, e->ev_out, 0));
  for (ib_grid_s *g : e->m) IB_CUDA(cudaStreamWaitEvent(g->s, e->ev_out, 0));
  return IB_OK;
}

}  // extern "C"
