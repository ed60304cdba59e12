/*
 * rve.h -- C ABI of librve: crack-length-controlled phase-field fracture on a periodic
 * voxel RVE, solved by an FFT-based monolithic Newton-Krylov method (arXiv 2412.17445,
 * Sec. 3.2 and Algorithm 2), on one NVIDIA GB300 (sm_103a).
 *
 * Conventions shared by every entry point
 *   - Every call returns an int status: RVE_OK (0) or a negative RVE_E_* code.  On error
 *     rve_last_error() describes it.  A failed call leaves the RVE in the state it had
 *     before the call (a failed crack increment rolls back to the last committed one).
 *   - Grids: nx * ny * nz voxels, voxel size h = 1, x fastest (index v = x + nx*(y + ny*z)).
 *     nz == 1 selects 2D plane strain (eps_zz = 0).  Each extent is 2^a 3^b, <= 4096.
 *   - Strain and stress fields are Mandel vectors (shear components times sqrt 2):
 *     2D m = 3 components (xx, yy, xy); 3D m = 6 (xx, yy, zz, yz, xz, xy).  A field of m
 *     components is stored component-major: comp k of voxel v at [k*n + v].
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA global memory of
 *     the device the RVE was created on.  The library never keeps a caller pointer: inputs
 *     are copied, outputs are written before the call returns (host) or in stream order
 *     (device).
 *   - An RVE handle is used by one host thread at a time.  All device work of a handle is
 *     issued on its stream (rve_set_stream; default: the legacy default stream).
 *   - Host arrays of floating-point state must be finite (rve_set_state rejects NaN / Inf
 *     with RVE_E_ARG before touching the device).
 *   - Test hook: the environment variable RVE_FAULT, read by rve_create / rve_load, injects
 *     a failure on the host side for that handle: "alloc:<k>" fails its k-th device
 *     allocation (rve_create returns RVE_E_OOM and frees what it had allocated);
 *     "krylov_breakdown" makes every BiCGStab solve of the handle break down (rho = 0), so
 *     increments end in RVE_E_NOCONV with the committed state kept.  Unset in production.
 */
#ifndef RVE_H
#define RVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RVE_OK 0
#define RVE_E_ARG (-1)      /* invalid argument or unsupported size                     */
#define RVE_E_OOM (-2)      /* device allocation failed                                 */
#define RVE_E_NOCONV (-3)   /* Newton did not converge; state rolled back               */
#define RVE_E_CUDA (-4)     /* CUDA runtime error (message in rve_last_error)           */
#define RVE_E_STATE (-5)    /* call not valid in the current state                      */
#define RVE_E_IO (-6)       /* file could not be read or written                        */

#define RVE_SPLIT_SPECTRAL 0 /* psi = g psi0+ + psi0- with the spectral split (Eq. PlusNegPsi) */
#define RVE_SPLIT_NONE 1     /* "isotropic" variant psi = g (psi0+ + psi0-) (Sec. 5.2)       */

#define RVE_GAMMA_ROTATED 0     /* Galerkin projection with Willot's rotated frequencies (Sec. 3.1) */
#define RVE_GAMMA_CONTINUOUS 1  /* ... with the continuous frequencies xi (Eq. GFourier); the     */
                                /* Nyquist component of xi is 0                                   */

#define RVE_CONSTRAINT_LENGTH 0  /* crack control prescribes the crack length Gamma (Eq. CrackLenght)  */
#define RVE_CONSTRAINT_ENERGY 1  /* ... the dissipated energy int G_c gamma_f (Eq. SystemDisc), with */
                                 /* gamma_f of Eq. newGammaFourier and G_c per voxel                 */

#define RVE_FP64 0           /* everything in float64                                          */
#define RVE_MIXED 1          /* float32 FFTs / Krylov, float64 residual, state and constraint  */

#define RVE_MAX_PHASES 16

typedef struct rve rve_t;

/* Problem description (Sec. 2, Table 2 style per-phase properties). */
typedef struct {
  int nx, ny, nz;          /* grid; nz == 1 -> 2D plane strain                           */
  int n_phases;            /* 1..RVE_MAX_PHASES                                          */
  const uint8_t *phase;    /* host, n voxels, phase id per voxel (copied)                */
  const double *E;         /* host, n_phases Young moduli                                 */
  const double *nu;        /* host, n_phases Poisson ratios                               */
  const double *Gc;        /* host, n_phases critical energy release rates                */
  double ell;              /* phase-field length scale, in voxels                         */
  double f[6];             /* load direction E_M = f E (Mandel, m entries used)           */
  int split;               /* RVE_SPLIT_SPECTRAL | RVE_SPLIT_NONE                          */
  int precision;           /* RVE_FP64 | RVE_MIXED                                         */
  double k_res;            /* residual stiffness k of g = (1-phi)^2 + k (0: plain AT2)       */
  double alpha;            /* Newton relaxation of Algorithm 2 (1 = none)                 */
  double newton_tol;       /* step / constraint tolerance of the Newton loop              */
  double krylov_tol;       /* relative BiCGStab tolerance                                 */
  int newton_max;          /* Newton iteration limit per increment                         */
  int krylov_max;          /* BiCGStab iteration limit per Newton iteration               */
  int gamma_op;            /* RVE_GAMMA_ROTATED (default) | RVE_GAMMA_CONTINUOUS          */
  int constraint;          /* RVE_CONSTRAINT_LENGTH (default) | RVE_CONSTRAINT_ENERGY      */
} rve_desc;

/* Fill a descriptor with the library defaults (spectral split, FP64, alpha 1,
 * newton_tol 1e-10, krylov_tol 1e-10, limits 50 / 4000).  For RVE_MIXED set krylov_tol
 * to about 1e-2: the float32 inner solve only has to contract the float64 Newton residual,
 * which alone sets the accuracy of the converged increment. */
void rve_desc_defaults(rve_desc *d);

/* Result of one increment. */
typedef struct {
  double E;                /* load factor E after the increment                         */
  double sigma[6];         /* macroscopic stress <sigma> (Mandel; shear x sqrt 2)        */
  double gamma;            /* crack length Gamma (Eq. CrackLenght)                       */
  double tau;              /* prescribed crack length                                    */
  int newton_iters;        /* Newton iterations                                           */
  int krylov_iters;        /* BiCGStab iterations summed over the Newton loop            */
  int applies;             /* operator applies (2 per BiCGStab iteration)                */
  double err;              /* final Newton error measure                                  */
  int cutbacks;            /* increments retried as two halves (cut-back), 0 normally     */
  int fallbacks;           /* RVE_MIXED: 1 if the increment was redone in float64 (below)   */
} rve_step;

/* Create an RVE (Sec. 3.1 discretisation).  Copies the phase map and properties to the
 * device and allocates all device memory of the solver.  Errors: RVE_E_ARG (sizes,
 * properties, precision), RVE_E_OOM, RVE_E_CUDA.  *out is NULL on error. */
int rve_create(const rve_desc *desc, rve_t **out);

/* Mark the initial crack (Sec. 4.1: the FFT model carries an initial crack one voxel thick;
 * Sec. 2.4: the elastic model cannot nucleate, so crack control starts from such a crack):
 * voxels with mask[v] != 0 hold phi = 1 as Dirichlet rows (Delta phi = 0 there).  host,
 * n bytes, x fastest, copied.  Valid only before the first increment (else RVE_E_STATE);
 * RVE_E_ARG if mask is NULL. */
int rve_set_notch(rve_t *h, const uint8_t *mask);

/* Start-up: strain-controlled steps E = 0 (phase-field profile of the notch), a probe load
 * and the load at which max 2 psi0+/(Gc/l) = beta; commits the history and tau_0 = the
 * constrained quantity of desc.constraint (Gamma, or int G_c gamma_f).
 * Called implicitly by the first rve_crack_increment; beta <= 0 selects 0.25. */
int rve_startup(rve_t *h, double beta, rve_step *out);

/* One crack-length increment (Algorithm 2 outer loop): tau += da, Newton with crack-length
 * control (Eq. System_CrackLength, Eq. LinearSyst_CrackCont), history commit (Eq. history).
 * da is in the units of desc.constraint: voxels of crack length (h = 1) under
 * RVE_CONSTRAINT_LENGTH, dissipated energy under RVE_CONSTRAINT_ENERGY (Eq. SystemDisc).
 * A failed Newton solve is retried as two committed half increments, recursively down to
 * da / 8 (out->cutbacks counts them).  Under RVE_MIXED an increment that still fails is
 * redone from the same committed state by a float64 twin of the handle (created on first
 * use, same stream, about twice the handle's device memory, freed with the handle;
 * out->fallbacks = 1; the counters then include both attempts); the environment variable
 * RVE_FP64_FALLBACK=0 switches this off.  out may be NULL.  RVE_E_NOCONV leaves the last
 * committed state. */
int rve_crack_increment(rve_t *h, double da, rve_step *out);

/* One strain-controlled monolithic increment to the load factor E_target (E_M = f E). */
int rve_strain_increment(rve_t *h, double E_target, rve_step *out);

/* Staggered strain-controlled increment (Algorithm 1): from the last committed state, at
 * E = E_target, alternate the mechanical solve at fixed phi and the phase-field solve at
 * fixed H = max(psi+, H^n) (each a Newton solve on its block of rows) until the summed
 * relative changes of eps_tilde and phi in a sweep are <= tol; then commit H.  In stable
 * regimes it reaches the state of rve_strain_increment.  *sweeps (may be NULL) receives the
 * sweeps used.  RVE_E_NOCONV after max_sweeps (state unchanged). */
int rve_staggered_increment(rve_t *h, double E_target, double tol, int max_sweeps, rve_step *out,
                            int *sweeps);

/* Macroscopic stress Sigma_M = <sigma>, the volume average of the microscopic stress (Sec. 2.2:
 * macroscopic strain and stress are volume averages, linked by the Hill-Mandel condition,
 * with E_M = f E), in Mandel form, and the load factor E of the committed state.  sigma
 * (6 host doubles; entries beyond m are 0) and E are host pointers, either may be NULL.
 * Re-evaluates the constitutive law on the device (blocking on the handle's stream), so a
 * later rve_apply / rve_apply_device needs rve_linearize again. */
int rve_get_macro_stress(const rve_t *h, double sigma[6], double *E);

/* Copy a field of the committed state to host memory (float64).  The unknowns of the
 * monolithic solver are q = {eps_tilde, phi, E} (Sec. 3.2, Eq. System_CrackLength); the
 * total strain is eps = eps_tilde + f E (Eq. stress_1a), H the history of Eq. history and
 * sigma the stress of Eq. OriSystem0a at the committed state:
 *   RVE_FIELD_EPS    m*n total strain eps = eps_tilde + f E
 *   RVE_FIELD_EPS_T  m*n strain fluctuation eps_tilde
 *   RVE_FIELD_PHI    n   phase field
 *   RVE_FIELD_H      n   history H
 *   RVE_FIELD_SIGMA  m*n stress
 * count is the number of doubles available at dst (RVE_E_ARG if too small). */
#define RVE_FIELD_EPS 0
#define RVE_FIELD_EPS_T 1
#define RVE_FIELD_PHI 2
#define RVE_FIELD_H 3
#define RVE_FIELD_SIGMA 4
int rve_get_fields(const rve_t *h, int which, double *dst, size_t count);

/* Overwrite the committed state (host float64 arrays; eps_tilde m*n, phi n, H n).  Used to
 * resume and by tests to linearise about a chosen point. */
int rve_set_state(rve_t *h, const double *eps_tilde, const double *phi, const double *H,
                  double E, double tau);

/* Autotuner of the FFT passes: times the operator apply (Eq. CrackLength_linearization)
 * on the device for candidate tiles (row pairs per x-pass block, kx columns per y/z-pass
 * block; fixed for float32 2D grids of at least 256 x 256) and then, for RVE_MIXED handles,
 * per axis whose length has no compile-time kernel, for candidate radix plans (radix-8 or
 * radix-4 stages, in either order), and keeps the fastest (RVE_FP64 handles keep the default
 * plan, so their rounding does not depend on timings).  Later handles of the same grid and precision in
 * the process reuse the choice.  Runs automatically before the first Newton solve of a
 * handle unless the environment sets RVE_AUTOTUNE=0; RVE_TILES="P,W" fixes the tiles and
 * RVE_RADIX_PLAN=<0..3> one plan variant on every axis (for tests). */
int rve_autotune(rve_t *h);

/* Issue all device work on this CUDA stream (a cudaStream_t cast to void*; NULL = default). */
int rve_set_stream(rve_t *h, void *stream);

/* Grid / layout queries. */
int rve_info(const rve_t *h, int *dim, int *m, long long *n, int *precision);

/* Checkpoint: the committed state, geometry, parameters, tiles and radix plans; a loaded
 * handle continues bit-exactly.  RVE_E_IO on a missing, truncated or foreign file. */
int rve_save(const rve_t *h, const char *path);
int rve_load(const char *path, rve_t **out);

void rve_destroy(rve_t *h);
const char *rve_last_error(const rve_t *h);   /* h may be NULL: last global error */

/* ---- Operator-level entry points (Sec. 3.2), for measurement and verification ---------
 * These act on the linearisation point = the current state (eps_tilde, phi, E, H^n).
 * rve_linearize evaluates the constitutive law (Eqs. PlusNegPsi, C_Calc, history),
 * the residual F = (F1, F2, F3) of Eq. System_CrackLength with control `control`
 * (RVE_CTRL_CRACK: F3 = Gamma - target; RVE_CTRL_STRAIN: F3 = E - target) and the
 * row scaling of the Newton system.  It must precede rve_apply / rve_residual calls. */
#define RVE_CTRL_CRACK 0
#define RVE_CTRL_STRAIN 1
int rve_linearize(rve_t *h, int control, double target);

/* Residual F of the last linearisation (unscaled, float64, host): F1 m*n, F2 n, F3 scalar. */
int rve_residual(const rve_t *h, double *F1, double *F2, double *F3);

/* Jacobian apply Delta F(q; Delta q) of Eq. CrackLength_linearization (unscaled, float64,
 * host in/out): dq_eps m*n, dq_phi n, dq_E scalar -> out_eps m*n, out_phi n, out_E. */
int rve_apply(rve_t *h, const double *dq_eps, const double *dq_phi, double dq_E,
              double *out_eps, double *out_phi, double *out_E);

/* Scaled Jacobian apply on device buffers in the Krylov precision (float for RVE_MIXED,
 * double for RVE_FP64): x and y hold c = m + 1 channels of n values (channel-major) and
 * xE / yE one double each.  y = S J x with the row scaling S of the linearisation.
 * Device pointers; runs on the RVE's stream; no synchronisation. */
int rve_apply_device(rve_t *h, const void *x, const double *xE, void *y, double *yE);

/* The scaled applies of rve_apply_device for count RVEs of one shape, precision and tile
 * schedule (the same tiles: RVEs tuned in one process share them), each FFT pass one launch
 * over all of them -- the grouping a batch of crack increments uses for its BiCGStab
 * iterations (Sec. 3.2).  x[i], xE[i], y[i], yE[i] are the device buffers of hs[i] as in
 * rve_apply_device.  1 <= count <= 8.  Runs on the stream of hs[0]; no synchronisation.
 * RVE_E_ARG if the RVEs differ in shape, precision or tiles, RVE_E_STATE if one of them is
 * not linearised. */
int rve_apply_device_batch(rve_t *const *hs, int count, const void *const *x, const double *const *xE,
                           void *const *y, double *const *yE);

/* Allocation-free variant of rve_apply_device.  No counterpart in the paper: it serves
 * callers that cannot allocate device memory when they call (code running during CUDA
 * graph capture, hosts whose device memory belongs to another allocator, service loops
 * that reserve everything at start-up).  Same arguments, result and stream as
 * rve_apply_device, but the spectral scratch and reduction partials come from one
 * file-scope device array of the library (16 MiB + 256 KiB, held by every GPU that loads
 * the library until the process exits) instead of the handle's buffers; the call performs
 * no cudaMalloc / cudaFree and calls no allocating library routine.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *     with that device current; make that first call before any stream capture.
 *   - Grids needing more scratch than the array holds are rejected with RVE_E_ARG (message
 *     in rve_last_error): spectral data 2 * p * (m+1) * ny * nz * (nx/2+1) bytes, p = 4
 *     (RVE_MIXED) or 8 (RVE_FP64).
 *   - Every call writes all scratch it later reads, so nothing needs to start at zero; the
 *     array keeps the last call's contents.
 *   - All calls share the one array: calls whose device work overlaps (different streams
 *     or host threads) race on it and give undefined results. */
int rve_apply_device_noalloc(rve_t *h, const void *x, const double *xE, void *y, double *yE);

/* Number of kernels the last rve_apply_device / rve_crack_increment launched. */
long long rve_kernel_launches(const rve_t *h);

/* ---- Batching (several RVEs advanced one increment each) ------------------------------
 * Advances every handle by one crack increment da[i].  Handles are independent; results
 * equal those of separate rve_crack_increment calls.  status[i] receives each status. */
int rve_batch_crack_increment(rve_t **hs, int count, const double *da, rve_step *out,
                              int *status);

/* Effective toughness of a crack-controlled run (Eq. JaviGc): G = (area / length) times the
 * area under the (E, Sigma:f) curve, trapezoid rule from the unloaded state (0, 0).  Host
 * arrays of n points; area = |Omega| (voxels), length = L_g, the crack length across the
 * cell.  Host arithmetic only. */
int rve_effective_toughness(const double *E, const double *sigma_f, int n, double area, double length,
                            double *G);

/* J-integral (Rice's contour integral in the x direction) of the committed state of a 2D
 * RVE: the energy release rate of a crack growing along +x, the post-processing check of
 * Sec. 4.2 that the crack-controlled path holds the dissipation near G_c times the
 * amplification factor of the appendix.
 *   J = sum over the rectangle of voxel centres (x0, y0)-(x1, y1), traversed once with
 *       outward normals n, of (W n_1 - sigma n . d_1 u) times the side length per voxel
 *       (the two end voxels of each side weighted 1/2), voxel size 1;
 *   W = g psi0+ + psi0- (spectral split) or g psi0 (RVE_SPLIT_NONE), sigma the stress of
 *       the constitutive law at eps = eps_tilde + f E;
 *   d_1 u_1 = E f_11 + eps~_11, d_1 u_2 = E f_21 + eps~_12 + w, with the rotation w of
 *       the periodic fluctuation displacement from the compatibility relations
 *       d_1 w = d_1 eps~_12 - d_2 eps~_11, d_2 w = d_1 eps~_22 - d_2 eps~_12, solved with the
 *       standard frequencies 2 pi k / N (Nyquist component 0) and zero mean.
 * 0 <= x0 < x1 < nx, 0 <= y0 < y1 < ny (x along the row, y across rows), else RVE_E_ARG;
 * RVE_E_ARG for 3D grids.  Float64 on the device, blocking on the handle's stream; *J is a
 * host double.  Uses the handle's spectral and stress scratch, so a later rve_apply_device
 * needs rve_linearize again. */
int rve_j_integral(rve_t *h, int x0, int y0, int x1, int y1, double *J);

/* Device bytes rve_create allocates for this descriptor (used for HBM-budget admission). */
int rve_footprint(const rve_desc *desc, long long *bytes);

/* ---- Serving: continuous batching of crack-increment requests --------------------------
 * A request = an RVE description + notch + n_increments crack-length increments of da.
 * Requests queue in arrival order.  While fewer than max_active run, the oldest queued
 * request whose footprint fits in the HBM budget beside the resident RVEs is admitted (any
 * request when none is resident), so a large request does not block smaller ones behind
 * it; a request overtaken max_active times stops all later admissions until it fits.
 * rve_server_create starts max_active worker threads, each with its own CUDA stream, that
 * run the admitted requests (start-up + increments; work of concurrent requests overlaps
 * on the device) and live until rve_server_destroy; an RVE stays resident until its
 * request completes.  Resident RVEs of equal shape and precision run their BiCGStab chunks
 * as grouped launches (one launch per pass for up to 4 RVEs, results identical to running
 * alone; RVE_SERVER_GROUPS=0 switches this off).  All copies of caller data are made by
 * rve_server_submit. */
typedef struct rve_server rve_server_t;
typedef struct {
  long long id;
  int status;              /* RVE_OK or the error of the request                            */
  int n_increments;        /* increments completed                                          */
  double E, sigma[6], gamma;  /* state after the last increment                             */
  double t_submit, t_start, t_end;  /* seconds on the server clock: queued, admitted, done  */
  long long footprint;     /* device bytes held while resident                              */
  char error[160];
} rve_result;
int rve_server_create(long long hbm_budget_bytes, int max_active, rve_server_t **out);
int rve_server_submit(rve_server_t *s, const rve_desc *desc, const uint8_t *notch, int n_increments,
                      double da, long long *id);   /* RVE_E_OOM if it can never fit the budget */
int rve_server_poll(rve_server_t *s, rve_result *res, int max, int *n);  /* completed requests */
int rve_server_drain(rve_server_t *s);             /* wait for every submitted request        */
int rve_server_stats(rve_server_t *s, long long *hbm_in_use, int *active, int *queued);
void rve_server_destroy(rve_server_t *s);          /* drains, then stops                      */

#ifdef __cplusplus
}
#endif
#endif /* RVE_H */
