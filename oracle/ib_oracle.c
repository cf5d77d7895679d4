/*
 * ib_oracle.c -- plain, slow, FP64 CPU oracle for the IB-GM time step of
 * Wiens & Stockie, "An Efficient Parallel Immersed Boundary Algorithm using a
 * Pseudo-Compressible Fluid Solver" (arxiv 1305.3976).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA implementation.
 *
 * Every function follows the paper's notation and order of operations:
 *   - discrete delta phi(r)             : Sec. 3.3, eq. (discretedelta)
 *   - MAC operators D_xx, G, D.         : Sec. 3.3 ("Spatial Finite Difference Operators")
 *   - D_s^+, D_s^-, force density        : Sec. 3.3 and Step 2a, eq. (forceDensityDefinition)
 *   - force connections (FC)             : Sec. 4.1, Fig. 3 (per-connection sigma)
 *   - interpolation / spreading          : Steps 1a and 2b
 *   - AB2 marker update, half position   : Steps 1b, 1c (forward Euler at n = 0)
 *   - skew-symmetric advection           : eq. (nonlinear) and the skew form that follows it
 *   - momentum + Douglas split           : Steps 3a-3d, eqs. (umacstep1), (umacstep2)
 *   - psi solve, pressure update         : Steps 3e-3f, eqs. (PenaltyStepPart1/2)
 *   - cyclic tridiagonal solve           : Sec. 4.2, block/Schur elimination,
 *                                          eqs. (LocalTriSystem), (SchurSystem), (SchurCorrection)
 *
 * Readings of points the paper leaves open (3D extension, skew-form stencil,
 * split-order rotation, rest length in the edge form) are documented next to
 * the code that implements them.
 *
 * Parity status: every exported function is pinned by a CPU test against a
 * closed form, an invariant or brute force (tests/test_oracle_*.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IBO_PI 3.14159265358979323846

typedef struct {
  int dim;       /* 2 or 3                                                 */
  int n[3];      /* cells per axis; n[2] == 1 when dim == 2                  */
  double H;      /* side of the periodic box [0,H]^d                         */
  double rho, mu, dt, chi;
  int kernel;    /* 0: 4-point kernel of eq. (discretedelta); 1: cosine      */
  int rotate;    /* 1: rotate the direction-split order with the step index */
  int schur_P;   /* number of blocks in the Schur line solve (>= 1)          */
  int scheme;    /* 0: the second-order GM variant of Sec. 3.4 (eqs.
                    PerturbNSE2-PerturbCorrection2); 1: the first-order
                    variant of Sec. 3.1, (eps/rho) A p + div u = 0 with
                    eps = dt (eqs. PerturbNSE-PerturbIncompressible)         */
} ibo_params;

typedef struct {
  double *u;      /* [dim][cells] MAC velocity u^n, component c on c-faces  */
  double *p;      /* [cells]  p^{n-1/2}                                     */
  double *psi;    /* [cells]  psi^{n-1/2}                                   */
  double *Nprev;  /* [dim][cells] N(u^{n-1})                                */
  double *X;      /* [nm][dim] marker positions X^n (unwrapped)            */
  double *Uprev;  /* [nm][dim] U^{n-1}                                      */
  int64_t nm;
  const int32_t *edges; /* [ne][2] force connections (a, b)                */
  const double *kappa;  /* [ne] spring constant of each connection         */
  const double *rest;   /* [ne] rest length of each connection             */
  int64_t ne;
  int64_t step;         /* n                                               */
} ibo_state;

/* ------------------------------------------------------------------------ */
/* grid helpers                                                              */

static long cells_of(const ibo_params *P) {
  return (long)P->n[0] * P->n[1] * (P->dim == 3 ? P->n[2] : 1);
}
static int nz_of(const ibo_params *P) { return P->dim == 3 ? P->n[2] : 1; }
static double h_of(const ibo_params *P, int a) { return P->H / P->n[a]; }

static long wrap(long i, long n) {
  long r = i % n;
  return r < 0 ? r + n : r;
}

/* linear index of cell/face (i,j,k) with periodic wrap; x fastest */
static long at(const ibo_params *P, long i, long j, long k) {
  long n0 = P->n[0], n1 = P->n[1], n2 = nz_of(P);
  return wrap(i, n0) + n0 * (wrap(j, n1) + n1 * wrap(k, n2));
}

/* index of the neighbour shifted by s along axis a */
static long shifted(const ibo_params *P, long i, long j, long k, int a, long s) {
  long q[3] = {i, j, k};
  q[a] += s;
  return at(P, q[0], q[1], q[2]);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3, eq. (discretedelta): the one-dimensional kernel phi(r).         */

double ibo_phi(int kernel, double r) {
  double a = fabs(r);
  if (kernel == 1) { /* cosine 4-point kernel: 1/4 (1 + cos(pi r / 2)) */
    return a < 2.0 ? 0.25 * (1.0 + cos(IBO_PI * r / 2.0)) : 0.0;
  }
  if (a < 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * r * r)) / 8.0;
  if (a < 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * r * r)) / 8.0;
  return 0.0;
}

/* Node offset (in cells) of MAC component c along axis a: the c-th velocity
 * component lives at i*h along its own axis and (i+1/2)*h along the others
 * (Sec. 3.2, Fig. 1). */
static double mac_offset(int c, int a) { return a == c ? 0.0 : 0.5; }

/* ------------------------------------------------------------------------ */
/* Step 1a: U_k = sum_{nodes} u(node) delta_h(node - X_k) h^d, where
 * delta_h h^d = prod_a phi((x_a(node) - X_a)/h_a).  The sum runs over a
 * window of 6 nodes per axis that contains the whole support |r| < 2; phi is
 * zero on the rest of the window, and on every node outside it.            */

void ibo_interp(const ibo_params *P, const double *u, const double *X, int64_t nm, double *U) {
  int d = P->dim;
  long cells = cells_of(P);
  for (int64_t k = 0; k < nm; ++k) {
    for (int c = 0; c < d; ++c) {
      long lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
      double h[3] = {1, 1, 1}, Xa[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) {
        h[a] = h_of(P, a);
        Xa[a] = X[k * d + a];
        long base = (long)floor(Xa[a] / h[a] - mac_offset(c, a));
        lo[a] = base - 2;
        hi[a] = base + 3;
      }
      double sum = 0.0;
      long kl = d == 3 ? lo[2] : 0, kh = d == 3 ? hi[2] : 0;
      for (long kk = kl; kk <= kh; ++kk)
        for (long jj = lo[1]; jj <= hi[1]; ++jj)
          for (long ii = lo[0]; ii <= hi[0]; ++ii) {
            long q[3] = {ii, jj, kk};
            double w = 1.0;
            for (int a = 0; a < d; ++a) {
              double xnode = ((double)q[a] + mac_offset(c, a)) * h[a];
              w *= ibo_phi(P->kernel, (xnode - Xa[a]) / h[a]);
            }
            if (w != 0.0) sum += u[c * cells + at(P, ii, jj, kk)] * w;
          }
      U[k * d + c] = sum;
    }
  }
}

/* Step 2b: f(node) = sum_k F_k delta_h(node - X_k) h_s.  The caller passes
 * the nodal force G_k = F_k h_s (trapezoid weight already applied), so
 * f(node) += G_k prod_a phi(...) / h^d.  Accumulates into f in marker order. */

void ibo_spread(const ibo_params *P, const double *X, const double *G, int64_t nm, double *f) {
  int d = P->dim;
  long cells = cells_of(P);
  double vol = 1.0;
  for (int a = 0; a < d; ++a) vol *= h_of(P, a);
  for (int64_t k = 0; k < nm; ++k) {
    for (int c = 0; c < d; ++c) {
      long lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
      double h[3] = {1, 1, 1}, Xa[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) {
        h[a] = h_of(P, a);
        Xa[a] = X[k * d + a];
        long base = (long)floor(Xa[a] / h[a] - mac_offset(c, a));
        lo[a] = base - 2;
        hi[a] = base + 3;
      }
      long kl = d == 3 ? lo[2] : 0, kh = d == 3 ? hi[2] : 0;
      for (long kk = kl; kk <= kh; ++kk)
        for (long jj = lo[1]; jj <= hi[1]; ++jj)
          for (long ii = lo[0]; ii <= hi[0]; ++ii) {
            long q[3] = {ii, jj, kk};
            double w = 1.0;
            for (int a = 0; a < d; ++a) {
              double xnode = ((double)q[a] + mac_offset(c, a)) * h[a];
              w *= ibo_phi(P->kernel, (xnode - Xa[a]) / h[a]);
            }
            if (w != 0.0) f[c * cells + at(P, ii, jj, kk)] += G[k * d + c] * w / vol;
          }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Step 2a, force connections of Sec. 4.1 (Fig. 3): every connection e joins
 * points a and b with spring constant kappa_e and rest length L_e; it pulls
 * a toward b with T = kappa_e (X_b - X_a)(1 - L_e/|X_b - X_a|) and b back by
 * -T.  Sums in edge order.  For a closed fiber of N_s points with
 * kappa_e = sigma/h_s and L_e = L h_s on consecutive points this equals
 * F_k h_s of Step 2a (checked against ibo_fiber_force_2d).                 */

void ibo_force_edges(int dim, double H, const double *X, int64_t nm, const int32_t *edges,
                     const double *kappa, const double *rest, int64_t ne, double *G) {
  for (int64_t i = 0; i < nm * dim; ++i) G[i] = 0.0;
  for (int64_t e = 0; e < ne; ++e) {
    int32_t a = edges[2 * e], b = edges[2 * e + 1];
    double D[3] = {0, 0, 0}, len2 = 0.0;
    for (int c = 0; c < dim; ++c) {
      D[c] = X[(int64_t)b * dim + c] - X[(int64_t)a * dim + c];
      /* a structure that closes on itself through the periodic box (the
       * cylinder of Sec. 6, whose ends join their periodic copies) is joined
       * through the nearest periodic image; for connections shorter than H/2
       * this changes nothing */
      D[c] -= H * round(D[c] / H);
      len2 += D[c] * D[c];
    }
    double scale = kappa[e];
    if (rest != NULL && rest[e] != 0.0) scale *= 1.0 - rest[e] / sqrt(len2);
    for (int c = 0; c < dim; ++c) {
      G[(int64_t)a * dim + c] += scale * D[c];
      G[(int64_t)b * dim + c] -= scale * D[c];
    }
  }
}

/* Step 2a written literally for one closed 2D fiber of ns points:
 * F_k = sigma D_s^- ( D_s^+ X_k (1 - L / |D_s^+ X_k|) ),
 * D_s^+ X_k = (X_{k+1} - X_k)/h_s,  D_s^- Y_k = (Y_k - Y_{k-1})/h_s.      */

void ibo_fiber_force_2d(const double *X, int64_t ns, double sigma, double L, double *F) {
  double hs = 1.0 / (double)ns;
  double *T = (double *)malloc(sizeof(double) * 2 * ns);
  for (int64_t k = 0; k < ns; ++k) {
    int64_t kp = (k + 1) % ns;
    double dx = (X[2 * kp] - X[2 * k]) / hs, dy = (X[2 * kp + 1] - X[2 * k + 1]) / hs;
    double norm = sqrt(dx * dx + dy * dy);
    double s = 1.0 - L / norm;
    T[2 * k] = dx * s;
    T[2 * k + 1] = dy * s;
  }
  for (int64_t k = 0; k < ns; ++k) {
    int64_t km = (k - 1 + ns) % ns;
    F[2 * k] = sigma * (T[2 * k] - T[2 * km]) / hs;
    F[2 * k + 1] = sigma * (T[2 * k + 1] - T[2 * km + 1]) / hs;
  }
  free(T);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3 difference operators.                                            */

/* D_aa q at every point: (q_{+1} - 2 q + q_{-1}) / h_a^2 */
void ibo_second_diff(const ibo_params *P, int a, const double *q, double *out) {
  double h = h_of(P, a);
  for (long k = 0; k < nz_of(P); ++k)
    for (long j = 0; j < P->n[1]; ++j)
      for (long i = 0; i < P->n[0]; ++i) {
        long c = at(P, i, j, k);
        out[c] = (q[shifted(P, i, j, k, a, 1)] - 2.0 * q[c] + q[shifted(P, i, j, k, a, -1)]) / (h * h);
      }
}

/* G^{C->E} p: component a on a-faces, (p_i - p_{i-1}) / h_a */
void ibo_gradient(const ibo_params *P, const double *p, double *g) {
  long cells = cells_of(P);
  for (int a = 0; a < P->dim; ++a) {
    double h = h_of(P, a);
    for (long k = 0; k < nz_of(P); ++k)
      for (long j = 0; j < P->n[1]; ++j)
        for (long i = 0; i < P->n[0]; ++i)
          g[a * cells + at(P, i, j, k)] = (p[at(P, i, j, k)] - p[shifted(P, i, j, k, a, -1)]) / h;
  }
}

/* D^{E->C} . u: sum_a (u_a at face i+1 - u_a at face i) / h_a */
void ibo_divergence(const ibo_params *P, const double *u, double *div) {
  long cells = cells_of(P);
  for (long k = 0; k < nz_of(P); ++k)
    for (long j = 0; j < P->n[1]; ++j)
      for (long i = 0; i < P->n[0]; ++i) {
        double s = 0.0;
        for (int a = 0; a < P->dim; ++a)
          s += (u[a * cells + shifted(P, i, j, k, a, 1)] - u[a * cells + at(P, i, j, k)]) / h_of(P, a);
        div[at(P, i, j, k)] = s;
      }
}

/* Skew-symmetric advection N(u) = 1/2 u.grad u + 1/2 div(u u), written with
 * the second-order staggered stencils of Morinishi et al. (1998) that the
 * paper cites (the paper prints no stencil).  For component c at its face
 * and each direction a:
 *   divergence half : [A+ * avg(u_c, +a) - A- * avg(u_c, -a)] / h_a
 *   advective half  : 1/2 [A+ (u_c(+a) - u_c)/h_a + A- (u_c - u_c(-a))/h_a]
 * where A+- is the a-velocity carried to the flux points half a cell above /
 * below the face along a: for a == c the average of u_c over its two faces,
 * otherwise the average of u_a over the two a-faces that straddle the c-face
 * along c.  The same A+- is used in both halves.                           */

void ibo_advection(const ibo_params *P, const double *u, double *N) {
  long cells = cells_of(P);
  int d = P->dim;
  for (int c = 0; c < d; ++c) {
    const double *uc = u + c * cells;
    for (long k = 0; k < nz_of(P); ++k)
      for (long j = 0; j < P->n[1]; ++j)
        for (long i = 0; i < P->n[0]; ++i) {
          long o = at(P, i, j, k);
          double total = 0.0;
          for (int a = 0; a < d; ++a) {
            double h = h_of(P, a);
            long op = shifted(P, i, j, k, a, 1), om = shifted(P, i, j, k, a, -1);
            double Ap, Am;
            if (a == c) {
              Ap = 0.5 * (uc[o] + uc[op]);
              Am = 0.5 * (uc[om] + uc[o]);
            } else {
              const double *ua = u + a * cells;
              long q[3] = {i, j, k};
              q[c] -= 1; /* the a-face one cell below along c */
              long o_c = at(P, q[0], q[1], q[2]);
              q[a] += 1;
              long op_c = at(P, q[0], q[1], q[2]);
              Ap = 0.5 * (ua[op] + ua[op_c]);
              Am = 0.5 * (ua[o] + ua[o_c]);
            }
            double div_half = (Ap * 0.5 * (uc[o] + uc[op]) - Am * 0.5 * (uc[om] + uc[o])) / h;
            double adv_half = 0.5 * (Ap * (uc[op] - uc[o]) / h + Am * (uc[o] - uc[om]) / h);
            total += 0.5 * (div_half + adv_half);
          }
          N[c * cells + o] = total;
        }
  }
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.2: periodic tridiagonal solve by block/Schur elimination.
 *
 * Row i of the cyclic system (indices mod n) reads
 *     c_i x_{i-1} + a_i x_i + b_i x_{i+1} = f_i .
 * The n unknowns are cut into P blocks; block p owns indices [s_p, s_{p+1})
 * with s_p = p n / P.  The first unknown of every block is an interface
 * unknown y_p = x_{s_p}; the rest of the block are interior unknowns x_p
 * that form the non-periodic tridiagonal block B_p.  Reordering gives
 *     [B E; F C][x; y] = [f; g],  S = C - F B^{-1} E,
 * and the solve is  B f* = f  (eq. LocalTriSystem, Thomas per block),
 * S y = g - F f*  (eq. SchurSystem, P x P), and x = f* - B^{-1} E y
 * (eq. SchurCorrection).  B^{-1}E and S depend only on the matrix, so they
 * are computed once in ibo_schur_setup (the paper precomputes them too).   */

typedef struct {
  int n, P;
  int *s;            /* [P+1] block starts                                   */
  double *a, *b, *c; /* [n] matrix rows                                      */
  double *cp;        /* [n] Thomas: modified super-diagonal per interior row */
  double *den;       /* [n] Thomas: pivot per interior row                   */
  double *Lv, *Rv;   /* [n] B^{-1}E columns: response to y_p / y_{p+1}       */
  double *S;         /* [P*P] Schur complement                               */
} ibo_schur;

/* Thomas forward/backward over the interior rows [lo, hi] of one block with
 * the pivots already stored in Z; rhs in f, result in x (both indexed by row). */
static void thomas_block(const ibo_schur *Z, int lo, int hi, const double *f, double *x) {
  double prev = 0.0;
  for (int i = lo; i <= hi; ++i) {
    double sub = (i == lo) ? 0.0 : Z->c[i];
    x[i] = (f[i] - sub * prev) / Z->den[i];
    prev = x[i];
  }
  for (int i = hi - 1; i >= lo; --i) x[i] -= Z->cp[i] * x[i + 1];
}

static void dense_solve(int P, double *A, double *rhs) {
  /* Gaussian elimination with partial pivoting on a small P x P system */
  for (int col = 0; col < P; ++col) {
    int piv = col;
    for (int r = col + 1; r < P; ++r)
      if (fabs(A[r * P + col]) > fabs(A[piv * P + col])) piv = r;
    if (piv != col) {
      for (int t = 0; t < P; ++t) {
        double tmp = A[col * P + t];
        A[col * P + t] = A[piv * P + t];
        A[piv * P + t] = tmp;
      }
      double tmp = rhs[col];
      rhs[col] = rhs[piv];
      rhs[piv] = tmp;
    }
    for (int r = col + 1; r < P; ++r) {
      double m = A[r * P + col] / A[col * P + col];
      for (int t = col; t < P; ++t) A[r * P + t] -= m * A[col * P + t];
      rhs[r] -= m * rhs[col];
    }
  }
  for (int r = P - 1; r >= 0; --r) {
    double s = rhs[r];
    for (int t = r + 1; t < P; ++t) s -= A[r * P + t] * rhs[t];
    rhs[r] = s / A[r * P + r];
  }
}

void ibo_schur_free(ibo_schur *Z) {
  if (!Z) return;
  free(Z->s); free(Z->a); free(Z->b); free(Z->c);
  free(Z->cp); free(Z->den); free(Z->Lv); free(Z->Rv); free(Z->S);
  free(Z);
}

ibo_schur *ibo_schur_setup(int n, int P, const double *a, const double *b, const double *c) {
  if (P < 1 || n < 2 * P) return NULL; /* every block needs an interior row */
  ibo_schur *Z = (ibo_schur *)calloc(1, sizeof(ibo_schur));
  Z->n = n;
  Z->P = P;
  Z->s = (int *)malloc(sizeof(int) * (P + 1));
  for (int p = 0; p <= P; ++p) Z->s[p] = (int)(((long)p * n) / P);
  Z->a = (double *)malloc(sizeof(double) * n);
  Z->b = (double *)malloc(sizeof(double) * n);
  Z->c = (double *)malloc(sizeof(double) * n);
  memcpy(Z->a, a, sizeof(double) * n);
  memcpy(Z->b, b, sizeof(double) * n);
  memcpy(Z->c, c, sizeof(double) * n);
  Z->cp = (double *)calloc(n, sizeof(double));
  Z->den = (double *)calloc(n, sizeof(double));
  Z->Lv = (double *)calloc(n, sizeof(double));
  Z->Rv = (double *)calloc(n, sizeof(double));
  Z->S = (double *)calloc((size_t)P * P, sizeof(double));
  /* Thomas pivots of each block B_p (interior rows s_p+1 .. s_{p+1}-1) */
  for (int p = 0; p < P; ++p) {
    int lo = Z->s[p] + 1, hi = Z->s[p + 1] - 1;
    for (int i = lo; i <= hi; ++i) {
      double sub = (i == lo) ? 0.0 : c[i];
      double cprev = (i == lo) ? 0.0 : Z->cp[i - 1];
      Z->den[i] = a[i] - sub * cprev;
      Z->cp[i] = (i == hi) ? 0.0 : b[i] / Z->den[i];
    }
  }
  /* B^{-1}E: column y_p enters the first interior row of block p through
   * c_{s_p+1}; column y_{p+1} enters its last interior row through
   * b_{s_{p+1}-1}. */
  double *e = (double *)calloc(n, sizeof(double));
  for (int p = 0; p < P; ++p) {
    int lo = Z->s[p] + 1, hi = Z->s[p + 1] - 1;
    for (int i = lo; i <= hi; ++i) e[i] = 0.0;
    e[lo] = c[lo];
    thomas_block(Z, lo, hi, e, Z->Lv);
    for (int i = lo; i <= hi; ++i) e[i] = 0.0;
    e[hi] = b[hi];
    thomas_block(Z, lo, hi, e, Z->Rv);
  }
  free(e);
  /* S = C - F B^{-1} E.  Interface row q couples to the last interior row of
   * block q-1 (through c_{s_q}) and the first interior row of block q
   * (through b_{s_q}).  Entry (B^{-1}E)[row in block p][col r] is Lv[row] if
   * r == p plus Rv[row] if r == p+1 (mod P). */
  for (int q = 0; q < P; ++q) {
    int sq = Z->s[q];
    int pm = (q - 1 + P) % P;
    int last_prev = Z->s[pm + 1] - 1; /* last interior row of block q-1 */
    int first_own = sq + 1;           /* first interior row of block q  */
    Z->S[q * P + q] += a[sq];
    /* contributions of block q-1 (columns q-1 and q) */
    Z->S[q * P + pm] -= c[sq] * Z->Lv[last_prev];
    Z->S[q * P + (pm + 1) % P] -= c[sq] * Z->Rv[last_prev];
    /* contributions of block q (columns q and q+1) */
    Z->S[q * P + q] -= b[sq] * Z->Lv[first_own];
    Z->S[q * P + (q + 1) % P] -= b[sq] * Z->Rv[first_own];
  }
  return Z;
}

/* Solve one cyclic system with a prepared Schur set-up; x may alias f. */
void ibo_schur_solve(const ibo_schur *Z, const double *f, double *x) {
  int n = Z->n, P = Z->P;
  double *fs = (double *)calloc(n, sizeof(double));
  double *y = (double *)malloc(sizeof(double) * P);
  double *Sw = (double *)malloc(sizeof(double) * P * P);
  /* eq. (LocalTriSystem): B_p f*_p = f_p on every block */
  for (int p = 0; p < P; ++p) thomas_block(Z, Z->s[p] + 1, Z->s[p + 1] - 1, f, fs);
  /* eq. (SchurSystem): S y = g - F f* */
  for (int q = 0; q < P; ++q) {
    int sq = Z->s[q];
    int pm = (q - 1 + P) % P;
    y[q] = f[sq] - Z->c[sq] * fs[Z->s[pm + 1] - 1] - Z->b[sq] * fs[sq + 1];
  }
  memcpy(Sw, Z->S, sizeof(double) * P * P);
  dense_solve(P, Sw, y);
  /* eq. (SchurCorrection): x_p = f*_p - B_p^{-1} E_p y */
  for (int p = 0; p < P; ++p) {
    double yl = y[p], yr = y[(p + 1) % P];
    for (int i = Z->s[p] + 1; i <= Z->s[p + 1] - 1; ++i) x[i] = fs[i] - Z->Lv[i] * yl - Z->Rv[i] * yr;
    x[Z->s[p]] = yl;
  }
  free(fs);
  free(y);
  free(Sw);
}

/* One general cyclic tridiagonal solve (set-up + solve); 0 on success. */
int ibo_cyclic_solve(int n, int P, const double *a, const double *b, const double *c,
                     const double *f, double *x) {
  ibo_schur *Z = ibo_schur_setup(n, P, a, b, c);
  if (!Z) return -1;
  ibo_schur_solve(Z, f, x);
  ibo_schur_free(Z);
  return 0;
}

/* (I - r D2) applied inverse along axis `axis` to every line of q, in place,
 * where D2 is the unit periodic second difference: row i reads
 * (1 + 2r) x_i - r x_{i-1} - r x_{i+1} = q_i  (eq. TriDiagX). */
int ibo_solve_lines(const ibo_params *P, int axis, double r, double *q) {
  int n = P->n[axis];
  int blocks = P->schur_P < 1 ? 1 : P->schur_P;
  double *a = (double *)malloc(sizeof(double) * n);
  double *b = (double *)malloc(sizeof(double) * n);
  double *c = (double *)malloc(sizeof(double) * n);
  for (int i = 0; i < n; ++i) {
    a[i] = 1.0 + 2.0 * r;
    b[i] = -r;
    c[i] = -r;
  }
  ibo_schur *Z = ibo_schur_setup(n, blocks, a, b, c);
  free(a); free(b); free(c);
  if (!Z) return -1;
  double *line = (double *)malloc(sizeof(double) * n);
  long dims[3] = {P->n[0], P->n[1], nz_of(P)};
  int o1 = (axis + 1) % 3, o2 = (axis + 2) % 3;
  for (long t2 = 0; t2 < dims[o2]; ++t2)
    for (long t1 = 0; t1 < dims[o1]; ++t1) {
      long q3[3];
      q3[o1] = t1;
      q3[o2] = t2;
      for (long i = 0; i < n; ++i) {
        q3[axis] = i;
        line[i] = q[at(P, q3[0], q3[1], q3[2])];
      }
      ibo_schur_solve(Z, line, line);
      for (long i = 0; i < n; ++i) {
        q3[axis] = i;
        q[at(P, q3[0], q3[1], q3[2])] = line[i];
      }
    }
  free(line);
  ibo_schur_free(Z);
  return 0;
}

/* Split order of time step n.  With rotation the order of step n is the
 * cyclic shift (n mod d) of (x, y[, z]); the paper rotates the order every
 * step without saying how, and on a periodic uniform grid the factors
 * commute, so any rotation gives the same result up to rounding. */
static void split_order(const ibo_params *P, int64_t n, int *order) {
  int d = P->dim;
  int shift = P->rotate ? (int)(n % d) : 0;
  for (int i = 0; i < d; ++i) order[i] = (i + shift) % d;
}

/* ------------------------------------------------------------------------ */
/* One IB-GM step (Sec. 3.4, Steps 1a-3f, with the n = 0 replacements).
 * Returns 0, or a negative value if a line solve cannot be set up.        */

int ibo_step(const ibo_params *P, ibo_state *S) {
  int d = P->dim;
  long cells = cells_of(P);
  int64_t nm = S->nm, n = S->step;
  double dt = P->dt, rho = P->rho, mu = P->mu;
  int rc = 0;

  double *U = (double *)calloc((size_t)(nm * d + 1), sizeof(double));
  double *Xnew = (double *)calloc((size_t)(nm * d + 1), sizeof(double));
  double *Xh = (double *)calloc((size_t)(nm * d + 1), sizeof(double));
  double *G = (double *)calloc((size_t)(nm * d + 1), sizeof(double));
  double *f = (double *)calloc((size_t)d * cells, sizeof(double));
  double *pstar = (double *)calloc((size_t)cells, sizeof(double));
  double *Nn = (double *)calloc((size_t)d * cells, sizeof(double));
  double *lap = (double *)calloc((size_t)cells, sizeof(double));
  double *gp = (double *)calloc((size_t)d * cells, sizeof(double));
  double *cur = (double *)calloc((size_t)d * cells, sizeof(double));
  double *div = (double *)calloc((size_t)cells, sizeof(double));
  double *avg = (double *)calloc((size_t)d * cells, sizeof(double));

  /* Step 1a */
  ibo_interp(P, S->u, S->X, nm, U);
  /* Steps 1b, 1c (forward Euler when n = 0) */
  for (int64_t i = 0; i < nm * d; ++i) {
    double vel = (n == 0) ? U[i] : 1.5 * U[i] - 0.5 * S->Uprev[i];
    Xnew[i] = S->X[i] + dt * vel;
    Xh[i] = 0.5 * (Xnew[i] + S->X[i]);
  }
  /* Step 2a */
  ibo_force_edges(d, P->H, Xh, nm, S->edges, S->kappa, S->rest, S->ne, G);
  /* Step 2b */
  ibo_spread(P, Xh, G, nm, f);
  /* Step 3a (p* = 0 when n = 0).  First-order variant: the momentum step
   * sees the latest pressure p^{n-1/2} itself. */
  for (long i = 0; i < cells; ++i)
    pstar[i] = (n == 0) ? 0.0 : (P->scheme == 1 ? S->p[i] : S->p[i] + S->psi[i]);
  /* Step 3b: rho((u* - u^n)/dt + N^{n+1/2}) = mu L u^n - G p* + f */
  ibo_advection(P, S->u, Nn);
  ibo_gradient(P, pstar, gp);
  for (int c = 0; c < d; ++c) {
    double *uc = S->u + c * cells;
    for (long i = 0; i < cells; ++i) cur[c * cells + i] = 0.0;
    for (int a = 0; a < d; ++a) {
      ibo_second_diff(P, a, uc, lap);
      for (long i = 0; i < cells; ++i) cur[c * cells + i] += mu * lap[i];
    }
    for (long i = 0; i < cells; ++i) {
      double Nhalf = (n == 0) ? Nn[c * cells + i] : 1.5 * Nn[c * cells + i] - 0.5 * S->Nprev[c * cells + i];
      double rhs = cur[c * cells + i] - gp[c * cells + i] + f[c * cells + i];
      cur[c * cells + i] = uc[i] + dt * (rhs / rho - Nhalf);
    }
  }
  /* Steps 3c-3d (and the z sweep in 3D): Douglas split, eqs. (umacstep1/2):
   * (I - a D_aa) u^{(a)} = u^{(a-1)} - a D_aa u^n,  a = mu dt / (2 rho). */
  double acoef = mu * dt / (2.0 * rho);
  int order[3];
  split_order(P, n, order);
  for (int s = 0; s < d; ++s) {
    int ax = order[s];
    double h = h_of(P, ax);
    for (int c = 0; c < d; ++c) {
      ibo_second_diff(P, ax, S->u + c * cells, lap);
      for (long i = 0; i < cells; ++i) cur[c * cells + i] -= acoef * lap[i];
      rc |= ibo_solve_lines(P, ax, acoef / (h * h), cur + c * cells);
    }
  }
  /* Step 3e: (1 - D_xx)(1 - D_yy)[(1 - D_zz)] psi = -rho/dt D.u^{n+1},
   * split into one sweep per axis (eqs. PenaltyStepPart1/2). */
  ibo_divergence(P, cur, div);
  for (long i = 0; i < cells; ++i) S->psi[i] = -rho / dt * div[i];
  for (int s = 0; s < d; ++s) {
    int ax = order[s];
    double h = h_of(P, ax);
    rc |= ibo_solve_lines(P, ax, 1.0 / (h * h), S->psi);
  }
  /* Step 3f: p^{n+1/2} = p^{n-1/2} + psi - chi mu D.(1/2 (u^{n+1} + u^n)).
   * First-order variant: the solve above is the pressure itself,
   * (dt/rho) A p^{n+1/2} = -D.u^{n+1}. */
  if (P->scheme == 1) {
    for (long i = 0; i < cells; ++i) S->p[i] = S->psi[i];
  } else {
    for (long i = 0; i < (long)d * cells; ++i) avg[i] = 0.5 * (cur[i] + S->u[i]);
    ibo_divergence(P, avg, div);
    for (long i = 0; i < cells; ++i) S->p[i] = S->p[i] + S->psi[i] - P->chi * mu * div[i];
  }

  /* roll the state forward */
  memcpy(S->u, cur, sizeof(double) * d * cells);
  memcpy(S->Nprev, Nn, sizeof(double) * d * cells);
  memcpy(S->Uprev, U, sizeof(double) * nm * d);
  memcpy(S->X, Xnew, sizeof(double) * nm * d);
  S->step = n + 1;

  free(U); free(Xnew); free(Xh); free(G); free(f); free(pstar); free(Nn);
  free(lap); free(gp); free(cur); free(div); free(avg);
  return rc ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Diagnostics (Sec. 5.1 volume conservation; discrete l2 norms of
 * eqs. ScalarDiscreteL2 / VectorDiscreteL2).                               */

/* Area enclosed by directed edges (a -> b) in 2D: 1/2 sum (x_a y_b - x_b y_a). */
double ibo_area_2d(const double *X, const int32_t *edges, int64_t ne) {
  double s = 0.0;
  for (int64_t e = 0; e < ne; ++e) {
    int32_t a = edges[2 * e], b = edges[2 * e + 1];
    s += X[2 * a] * X[2 * b + 1] - X[2 * b] * X[2 * a + 1];
  }
  return 0.5 * s;
}

/* Signed volume enclosed by oriented triangles: 1/6 sum X_a . (X_b x X_c). */
double ibo_volume_3d(const double *X, const int32_t *tris, int64_t nt) {
  double s = 0.0;
  for (int64_t t = 0; t < nt; ++t) {
    const double *A = X + 3 * tris[3 * t], *B = X + 3 * tris[3 * t + 1], *C = X + 3 * tris[3 * t + 2];
    s += A[0] * (B[1] * C[2] - B[2] * C[1]) - A[1] * (B[0] * C[2] - B[2] * C[0]) +
         A[2] * (B[0] * C[1] - B[1] * C[0]);
  }
  return s / 6.0;
}

/* Elastic energy of the force connections: sum 1/2 kappa (|X_b - X_a| - L)^2 */
double ibo_elastic_energy(int dim, const double *X, const int32_t *edges, const double *kappa,
                          const double *rest, int64_t ne) {
  double s = 0.0;
  for (int64_t e = 0; e < ne; ++e) {
    double len2 = 0.0;
    for (int c = 0; c < dim; ++c) {
      double dd = X[(int64_t)edges[2 * e + 1] * dim + c] - X[(int64_t)edges[2 * e] * dim + c];
      len2 += dd * dd;
    }
    double ext = sqrt(len2) - (rest ? rest[e] : 0.0);
    s += 0.5 * kappa[e] * ext * ext;
  }
  return s;
}
