/*
 * ib_gb300.h -- C ABI of the GB300 (sm_103a) implementation of one IB-GM time
 * step of Wiens & Stockie, "An Efficient Parallel Immersed Boundary Algorithm
 * using a Pseudo-Compressible Fluid Solver" (arxiv 1305.3976), Sec. 3.4.
 *
 * Conventions shared by every entry point
 *   - Return IB_OK (0) or a negative IB_ERR_* code; ib_last_error() gives a
 *     message for the calling thread's most recent failure.  No entry point
 *     aborts, traps or prints.
 *   - Plain pointers only.  A pointer argument is host memory unless its
 *     `*_on_device` flag (or the entry point) says it is a CUDA device
 *     pointer of the current device.
 *   - Inputs are copied: the caller keeps ownership of every buffer it passes
 *     and may free it when the call returns.  The library owns the device
 *     state behind an ib_grid_t and frees it in ib_destroy_grid.
 *   - Work is stream-ordered on the stream given in ib_grid_desc.stream (a
 *     cudaStream_t; NULL means the legacy default stream).  Calls that return
 *     data to host memory synchronise that stream before returning.
 *   - Fields are stored SoA, x fastest: index i + n0 (j + n1 k).  Velocity
 *     component c lives on the c-faces of the MAC grid (Sec. 3.2, Fig. 1):
 *     u at (i h, (j+1/2) h, (k+1/2) h), v at ((i+1/2) h, j h, (k+1/2) h),
 *     w at ((i+1/2) h, (j+1/2) h, k h); p and psi at cell centres.
 *   - Markers are FP64, array-of-structs [n_markers][dim], unwrapped (the
 *     periodic wrap is applied to grid indices only).
 */
#ifndef IB_GB300_H
#define IB_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  IB_OK = 0,
  IB_ERR_ARG = -1,       /* invalid argument (null pointer, size, range)       */
  IB_ERR_OOM = -2,       /* device or host allocation failed                    */
  IB_ERR_CUDA = -3,      /* a CUDA runtime call failed (see ib_last_error)      */
  IB_ERR_NONFINITE = -4, /* a NaN or Inf was found in the state                 */
  IB_ERR_TIMEOUT = -5,   /* a bounded device-side wait ran out (ib_diagnostics) */
  IB_ERR_STATE = -6      /* call not allowed in the grid's current state        */
};

enum { IB_FP32 = 0, IB_FP64 = 1 };                 /* field precision          */
enum { IB_DELTA_PESKIN4 = 0, IB_DELTA_COS4 = 1 };  /* 1D kernel phi(r)         */
enum { IB_GM2 = 0, IB_GM1 = 1 };                   /* pseudo-compressibility   */

/* field selection bits for ib_read_fields */
enum {
  IB_FIELD_U = 1, IB_FIELD_V = 2, IB_FIELD_W = 4,
  IB_FIELD_P = 8,    /* p^{n-1/2} after n steps                       */
  IB_FIELD_PSI = 16, /* psi^{n-1/2}                                   */
  IB_FIELD_DIV = 32  /* D.u^n (cell centres)                          */
};

typedef struct ib_grid_s *ib_grid_t;

/* Problem description (Sec. 3.2-3.4).
 *   dim          2 or 3.
 *   n[3]         cells per axis, each 8 <= n <= 512 (n[2] ignored in 2D);
 *                h_a = H / n[a].
 *   H            side of the periodic box [0,H]^d.
 *   rho, mu      density and dynamic viscosity (eq. NSE).
 *   dt           time step (also the perturbation parameter epsilon).
 *   chi          weight of the pressure update, Step 3f (the paper uses 0.6).
 *   precision    IB_FP32 or IB_FP64 fields; markers are always FP64.
 *   kernel       IB_DELTA_PESKIN4 (eq. discretedelta) or IB_DELTA_COS4
 *                (phi = (1 + cos(pi r / 2)) / 4 on |r| < 2).
 *   rotate_split 1: step n applies the direction-split factors in the order
 *                cyclically shifted by n mod dim (Sec. 4.1); 0: x, y(, z).
 *   stream       cudaStream_t the grid works on (NULL: default stream).
 *   scheme       IB_GM2 (0): the second-order Guermond-Minev variant the paper
 *                uses (Sec. 3.1 eqs. PerturbNSE2-PerturbCorrection2; Sec. 3.4
 *                Steps 3a, 3e, 3f).  IB_GM1 (1): the first-order variant of
 *                Sec. 3.1, (eps/rho) A p + D.u = 0 with eps = dt: Step 3a
 *                uses p* = p^{n-1/2}, the solve of Step 3e gives p^{n+1/2}
 *                itself, chi is not used.                                   */
typedef struct {
  int dim;
  int n[3];
  double H, rho, mu, dt, chi;
  int precision;
  int kernel;
  int rotate_split;
  void *stream;
  int scheme;
} ib_grid_desc;

/* FP64 diagnostics (Sec. 5.1 volume conservation; discrete l2 norms of
 * eqs. ScalarDiscreteL2 / VectorDiscreteL2). */
typedef struct {
  double volume;   /* area (2D, from the oriented edge loops) or volume (3D,
                      from the oriented triangles passed to ib_add_fiber)      */
  double div_l2;   /* (h^d sum (D.u)^2)^{1/2}                                 */
  double div_max;  /* max |D.u|                                               */
  double kinetic;  /* 1/2 rho h^d sum |u|^2                                   */
  double elastic;  /* sum over connections 1/2 kappa (|X_b - X_a| - L)^2 at X^n */
  int64_t step;    /* n                                                      */
} ib_diag;

/* Create a grid with u = 0, p = psi = 0 and no markers (Sec. 3.4, n = 0).
 * Allocates (3 dim + 3) fields of n0 n1 n2 elements on the current device.
 * Errors: IB_ERR_ARG (bad desc), IB_ERR_OOM, IB_ERR_CUDA. */
int ib_create_grid(const ib_grid_desc *desc, ib_grid_t *out);

/* Append one structure made of points and force connections (Sec. 4.1,
 * Fig. 3; Step 2a): connection e joins points edges[2e], edges[2e+1] (indices
 * local to this call, 0 <= index < n_markers) and pulls them together with
 *   T_e = kappa[e] (X_b - X_a) (1 - rest_len[e] / |X_b - X_a|),
 * the difference taken through the nearest periodic image.  A closed 2D fiber
 * of N_s points with kappa = sigma / h_s and rest_len = L h_s reproduces the
 * paper's F_k h_s.  rest_len may be NULL (all zero).  tris (optional, 3D:
 * [n_tris][3] outward-oriented triangles; 2D: ignored, the directed edges give
 * the area) feed ib_diagnostics.  Every array may be host memory or device
 * memory of the current device (told apart by cudaPointerGetAttributes; device
 * arrays are copied to the host on the grid's stream, which the call then
 * synchronises).  Only allowed before the first step.  fiber_id_out (optional) receives the structure's
 * index.  Errors: IB_ERR_ARG, IB_ERR_STATE, IB_ERR_OOM, IB_ERR_CUDA. */
int ib_add_fiber(ib_grid_t g, const double *X0, int64_t n_markers, const int32_t *edges,
                 const double *kappa, const double *rest_len, int64_t n_edges,
                 const int32_t *tris, int64_t n_tris, int32_t *fiber_id_out);

/* Set velocity component comp (0..dim-1) from n0 n1 n2 elements of the
 * grid's precision (host memory, or device memory if on_device).  Only
 * allowed before the first step.  Errors: IB_ERR_ARG, IB_ERR_STATE, IB_ERR_CUDA. */
int ib_set_velocity(ib_grid_t g, int comp, const void *src, int on_device);

/* Advance n_steps IB-GM steps (Sec. 3.4, Steps 1a-3f; the first step uses the
 * n = 0 replacements).  Asynchronous on the grid's stream.
 * Errors: IB_ERR_ARG (n_steps < 0), IB_ERR_CUDA. */
int ib_step(ib_grid_t g, int n_steps);

/* Copy the fields selected by field_mask, in the bit order U, V, W, P, PSI,
 * DIV, each n0 n1 n2 elements of the grid's precision, back to back into dst
 * (bytes must equal the total).  Host dst: the call returns when the data is
 * there; device dst: stream-ordered.  Errors: IB_ERR_ARG, IB_ERR_CUDA. */
int ib_read_fields(ib_grid_t g, unsigned field_mask, void *dst, size_t bytes, int dst_on_device);

/* Copy the marker positions X^n ([n][dim] FP64, all structures in the order
 * they were added) to X; n must equal the total marker count.
 * Errors: IB_ERR_ARG, IB_ERR_CUDA. */
int ib_read_markers(ib_grid_t g, double *X, int64_t n, int dst_on_device);

/* Replace the marker positions X^n (for example by a host-side structure
 * model coupled to the fluid); U^{n-1} is kept.  Errors: IB_ERR_ARG, IB_ERR_CUDA. */
int ib_set_markers(ib_grid_t g, const double *X, int64_t n, int src_on_device);

/* FP64 diagnostics of the current state; synchronises the grid's stream.
 * Returns IB_ERR_NONFINITE (after filling *out) if any value is NaN or Inf,
 * and IB_ERR_TIMEOUT if, since the last such report, a kernel of this
 * process gave up a bounded wait for its staged copies (results of that
 * launch are then not to be trusted). */
int ib_diagnostics(ib_grid_t g, ib_diag *out);

/* Release every device and host resource of the grid. */
int ib_destroy_grid(ib_grid_t g);

/* Static text for an IB_* code; message of the calling thread's last error. */
const char *ib_error_string(int code);
const char *ib_last_error(void);

/* Ensembles of independent grids (each with its own size, parameters and
 * structures) advanced together.  Members of the same precision and size form
 * a size class, split into groups of at most 4; every kernel of a step
 * (Sec. 3.4, Steps 1a-3f) is one batched launch per group that walks the
 * group's member table, the groups run side by side, and a whole ensemble
 * step is one CUDA graph launch.  The paper runs one problem at a time; this batches
 * many.  Within a group the line solves use the register kernels with the
 * shape the group's first member chose (ib_sweep_config), so an ensemble
 * member agrees with the same grid stepped alone to rounding.
 *   ib_create_ensemble: members are existing grids (the ensemble does not own
 *     them) that all have the same dim, the same rotate_split and the same
 *     step count; their structures must already be added.  stream: as in
 *     ib_grid_desc.
 *   ib_ensemble_step: advances every member by n_steps (Sec. 3.4), ordered
 *     after earlier work on the members; afterwards the members can be read
 *     or stepped on their own.
 * Errors: IB_ERR_ARG, IB_ERR_STATE (mismatched members), IB_ERR_CUDA. */
typedef struct ib_ensemble_s *ib_ensemble_t;
int ib_create_ensemble(const ib_grid_t *members, int n_members, void *stream, ib_ensemble_t *out);
int ib_ensemble_step(ib_ensemble_t e, int n_steps);
int ib_destroy_ensemble(ib_ensemble_t e);

/* Batched constant-coefficient cyclic tridiagonal solve along one axis
 * (Sec. 4.2, eq. TriDiagX): every line along `axis` of the n0 x n1 x n2 field
 * `in` is replaced by the solution x of
 *   (1 + 2r) x_i - r x_{i-1} - r x_{i+1} = b_i   (indices mod n[axis]),
 * written to `out` (device pointers of the given precision; out may equal in).
 * dim 2 ignores n[2]; 8 <= n[a] <= 512.  r >= 0.  Stream-ordered on `stream`.
 * Errors: IB_ERR_ARG, IB_ERR_CUDA. */
int ib_cyclic_solve_lines(int precision, int dim, const int n[3], int axis, double r,
                          const void *in, void *out, void *stream);

/* The direction-split operator of the paper's Poisson comparison (Sec. 6.1,
 * eq. PoissonGMProblem) and of Step 3e: solves
 *   (I - r_0 D2_x)(I - r_1 D2_y)[(I - r_2 D2_z)] psi = f
 * with D2 the unit periodic second difference (for Step 3e, r_a = 1/h_a^2)
 * as one sweep per axis: f (device) -> psi (device; may equal f).
 * Errors: IB_ERR_ARG, IB_ERR_CUDA. */
int ib_split_solve(int precision, int dim, const int n[3], const double r[3], const void *f,
                   void *psi, void *stream);

/* Allocation-free variant of ib_split_solve.  The paper has no counterpart;
 * it exists for callers that cannot allocate device memory: processes whose
 * device memory belongs to another allocator (a framework's caching
 * allocator, a budget fixed at start-up) and latency-critical loops that must
 * not call cudaMalloc because it synchronises the device.  ib_split_solve
 * allocates a small table of powers lam^k per (n, r) on first use; this
 * variant keeps those tables in one fixed array inside the library (file-scope
 * __device__ storage of about 25 KB that every GPU loading the library holds
 * until the process exits) and calls no cudaMalloc, cudaFree or other
 * allocating routine.  Same arguments, layout, result and stream ordering as
 * ib_split_solve.
 *   - Line lengths are limited to IB_NOALLOC_MAX_N (= 512); a larger n[a]
 *     returns IB_ERR_ARG with a message naming the limit.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current, and again after the
 *     device's context was created anew (e.g. after cudaDeviceReset); make
 *     that first call before any stream capture.  Devices 0 .. 63 are
 *     supported; a call on a device with a higher index returns IB_ERR_ARG.
 *   - Every call rewrites the shared array before its solves read it, so no
 *     state carries over between calls, but calls whose work overlaps on the
 *     GPU (different streams, or different host threads) race on the array:
 *     order them on one stream.
 * Errors: IB_ERR_ARG, IB_ERR_CUDA. */
#define IB_NOALLOC_MAX_N 512
int ib_split_solve_noalloc(int precision, int dim, const int n[3], const double r[3], const void *f,
                           void *psi, void *stream);

/* The line-solve configuration a grid chose for `axis` (0..dim-1).  On its
 * first step (or first call that needs the device state) a grid times every
 * candidate configuration of its sweeps per axis on its own scratch fields, in
 * each of the step's five sweep roles (plain momentum sweep, last momentum
 * sweep with u^n + e, plain psi sweep, first psi sweep with the divergence,
 * last psi sweep with p + psi), and keeps the fastest per role; this call
 * reports the plain momentum sweep's.  cfg[4] receives: the configuration
 * id, then for y/z lines the vector width (adjacent x lines per thread), the
 * chunk length and the warps per line, or for x lines 1, the warps per CTA (8)
 * and the cap on CTAs per SM.  Errors: IB_ERR_ARG, IB_ERR_CUDA. */
int ib_sweep_config(ib_grid_t g, int axis, int cfg[4]);

/* Use line-solve configuration `id` (an id that ib_sweep_config reported for
 * a grid of the same size and precision) for every sweep role along `axis`
 * instead of timing the candidates (the sweeps with a prologue or epilogue
 * take the library's default shape where `id` is the TMA kernel, 11), e.g. to
 * reproduce a run's choice under a profiler, where timings are distorted.  Only before the first step.  Errors: IB_ERR_ARG (axis, or
 * id not a candidate for this grid), IB_ERR_STATE (grid already stepped). */
int ib_fix_sweep_config(ib_grid_t g, int axis, int id);

/* Marker re-sorting (no counterpart in the paper, whose Lagrangian data
 * migrate between processors instead; Sec. 4.1).  Internally the markers are
 * numbered in the Morton order of their positions, so that neighbouring
 * threads of interpolation and spreading touch neighbouring grid nodes; the
 * numbering is taken from the initial positions, and structures that travel
 * (Sec. 6.3: ellipses carried through the periodic box) can be re-numbered by
 * their current positions.  Results are unchanged up to the summation order
 * of the spreading atomics, and ib_read_markers / ib_set_markers /
 * ib_save_state / ib_adjoint_run keep using the caller's order.
 *   ib_resort_markers: re-number now (host-side sort of the current
 *     positions; synchronises the grid's stream).
 *   ib_set_resort_interval: re-number before every step n with n % every == 0
 *     (n > 0) inside ib_step (each time synchronising the stream); 0 (the
 *     default) never.  Ensemble steps and ib_adjoint_run do not re-number.
 * Errors: IB_ERR_ARG (null grid, every < 0), IB_ERR_CUDA. */
int ib_resort_markers(ib_grid_t g);
int ib_set_resort_interval(ib_grid_t g, int every);

/* Run n_steps steps with every kernel launched on its own and timed by CUDA
 * events on the grid's stream; kernel_ms[i] receives the total milliseconds
 * of kernel slot i (at most max_kernels slots, *n_kernels gets the count) and
 * ib_kernel_name(i) its name.  Advances the state like ib_step.
 * Errors: IB_ERR_ARG, IB_ERR_CUDA. */
int ib_profile_step(ib_grid_t g, int n_steps, float *kernel_ms, int max_kernels, int *n_kernels);
const char *ib_kernel_name(int slot);

/* Discrete adjoint of n_steps IB-GM steps with respect to the connection
 * stiffnesses (no counterpart in the paper, which states no optimisation
 * problem; the map it differentiates is the step of Sec. 3.4, Steps 1a-3f,
 * with the connection force of Sec. 4.1, Fig. 3 at zero rest length).
 *   Advances g by n_steps exactly as ib_step(g, n_steps) does and leaves it
 *   in that state.  *loss receives sum_k |X_k - X_target_k|^2 over the final
 *   marker positions and dkappa[e] = d loss / d kappa_e for every connection
 *   e, in the order the connections were added by ib_add_fiber (all fibers,
 *   concatenated).  The gradient is the exact transpose of the discrete step
 *   (weight derivatives of the delta kernel, AB2 histories, the Jacobian of
 *   the skew-symmetric advection), up to rounding.
 *   X_target: host, [n_markers][dim] FP64 in the caller's marker order;
 *   loss: host double; dkappa: host, [n_edges] FP64.
 *   checkpoint_every >= 1: the state (2 dim + 3 fields, X, U^{n-1}) is kept
 *   every that many steps; each segment is run forward twice (once to
 *   checkpoint, once to record u, X, U^{n-1} of its steps) and then backward.
 *   Device memory: (ceil(n_steps / checkpoint_every) + 1) states, plus
 *   checkpoint_every * dim fields of tape, plus 4 dim + 4 adjoint fields,
 *   allocated on entry and freed before return.
 * Synchronises the grid's stream.  Errors: IB_ERR_ARG (null pointer, n_steps
 * < 0, checkpoint_every < 1, a non-zero rest length), IB_ERR_OOM (checkpoints
 * do not fit), IB_ERR_NONFINITE (non-finite final position), IB_ERR_CUDA. */
int ib_adjoint_run(ib_grid_t g, int n_steps, int checkpoint_every, const double *X_target, double *loss,
                   double *dkappa);

/* Checkpoint / resume (the paper has none): the complete state S^n of a grid
 * -- u, p^{n-1/2}, psi^{n-1/2}, N(u^{n-1}), D.u^n, the marker positions X^n,
 * U^{n-1} and the step count n -- as a host byte image, so that a grid
 * loaded from it continues exactly as the saved one would (Sec. 3.4: the
 * step reads nothing else).  Layout: a 64-byte header (magic "IBGMSTAT",
 * version, dim, n[3], precision, scheme, marker and connection counts, n),
 * the fields u[0..dim), p, psi, N[0..dim), D.u, each n0 n1 n2 elements of the
 * grid's precision in grid order, X as [n_markers][dim] FP64 and U^{n-1} as
 * [n_markers][dim] of the field precision, markers in the caller's order.
 *   ib_state_size: bytes of the image.
 *   ib_save_state: writes the image to host memory dst (bytes must match);
 *     synchronises the grid's stream.
 *   ib_load_state: replaces the grid's state by the image at host memory src.
 *     The grid must have the same dim, n, precision, scheme and the same
 *     structures added (marker and connection counts are checked; the
 *     connections themselves are the caller's to match).
 * Errors: IB_ERR_ARG (null pointer, size, image of another grid), IB_ERR_CUDA. */
int ib_state_size(ib_grid_t g, size_t *bytes);
int ib_save_state(ib_grid_t g, void *dst, size_t bytes);
int ib_load_state(ib_grid_t g, const void *src, size_t bytes);

/* Self-test of the bounded device waits (no counterpart in the paper).  The
 * kernels that stage data with bulk tensor copies wait on mbarriers for at
 * most 1 s; when a wait runs out they set a process-wide flag, which
 * ib_diagnostics reports as IB_ERR_TIMEOUT, and return.  This call launches
 * one CTA that arms an mbarrier for bytes no copy will deliver and waits with
 * a 1 ms limit, so the wait runs out: *timed_out receives the flag (1 when the
 * mechanism works), which is then cleared.  The CUDA context stays usable.
 * Synchronises `stream` (a cudaStream_t; NULL: default stream).
 * Errors: IB_ERR_ARG, IB_ERR_CUDA. */
int ib_selftest_wait_timeout(void *stream, int *timed_out);

/* Throughput probes of the current GPU (no counterpart in the paper), the
 * ceilings of the step's kernels that are not bound by HBM bandwidth:
 *   IB_PEAK_FP64_FMA   FP64 fused multiply-adds, in FLOP/s (2 per FMA): the
 *                      FP64 right-hand side and line solves;
 *   IB_PEAK_FP32_FMA   the same in FP32;
 *   IB_PEAK_L2_ATOMIC  float atomic adds without return, each warp instruction
 *                      on 32 consecutive floats of an L2-resident 16 MB
 *                      buffer, in updates/s: spreading (Step 2b).
 * Runs 3 warm-up and 5 timed launches on `stream` (a cudaStream_t; NULL:
 * default stream), timed by CUDA events, and writes the best rate to *value
 * (host).  Allocates and frees a 16 MB scratch buffer; synchronises the
 * stream.  Errors: IB_ERR_ARG (kind, null value), IB_ERR_OOM, IB_ERR_CUDA. */
enum { IB_PEAK_FP64_FMA = 0, IB_PEAK_FP32_FMA = 1, IB_PEAK_L2_ATOMIC = 2 };
int ib_measure_peak(int kind, void *stream, double *value);

#ifdef __cplusplus
}
#endif

#endif /* IB_GB300_H */
