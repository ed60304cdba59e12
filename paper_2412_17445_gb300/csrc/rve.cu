// Host driver and C ABI of librve (include/rve.h).
//
// One RVE = one set of device buffers.  A crack increment (Algorithm 2) is a host loop of
// Newton iterations; each iteration evaluates the float64 constitutive law and residual on
// the device, then runs BiCGStab entirely on the device (scalars in device memory, the host
// only polls a "done" flag every few iterations), then applies the Newton update.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <algorithm>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <map>
#include <mutex>
#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rve.h"
#include "post.cuh"
#include "rve_internal.h"
#include "rve_kern.cuh"

// ---- kernels defined in kernels_fft.cu / kernels_pw.cu -----------------------------------
template <typename T, int M, int NL, int PC, int MODE> __global__ void k_xfwd_apply(const __grid_constant__ ApplyGroup<T>, FftPlan, int);
template <typename T, int M, int NL, int PC, int MODE> __global__ void k_xinv_apply(const __grid_constant__ ApplyGroup<T>, FftPlan, int);
template <typename T, int M, int MODE, int NL> __global__ void k_col(const __grid_constant__ ColGroup<T>);

// Pass kernels by line length: compile-time lengths where instantiated (kernels_fft_<N>.cu:
// 2D at 48, 64, 96, 128, 192, 256, 384, 512, 1024; 3D at 48, 64, 96, 128), the runtime-length
// kernels otherwise.
template <typename T> using RowKernel = void (*)(const __grid_constant__ ApplyGroup<T>, FftPlan, int);
template <typename T> using ColKernel = void (*)(const __grid_constant__ ColGroup<T>);

// a launch over one RVE is a group of one member
template <typename T>
static ApplyGroup<T> solo(const ApplyArgs<T> &a) {
  ApplyGroup<T> g;
  memset((void *)&g, 0, sizeof g);
  g.m[0] = a;
  return g;
}
template <typename T>
static ColGroup<T> solo_col(const ColArgs<T> &a) {
  ColGroup<T> g;
  memset((void *)&g, 0, sizeof g);
  g.base = a;
  g.spec[0] = a.spec;
  g.ks[0] = a.ks;
  return g;
}
template <typename TK>
static KvGroup<TK> solo_kv(const KvArgs<TK> &a) {
  KvGroup<TK> g;
  memset((void *)&g, 0, sizeof g);
  g.m[0] = a;
  return g;
}
// column lengths of the fused 2D column pass (transposed spectral scratch)
static const int kCtLengths[5] = {64, 128, 256, 512, 1024};

// x-pass kernel for line length N: a compile-time length where one is built, else the
// runtime-length kernel; the float32 2D passes with P = 1 or 2 row pairs per block come
// specialised on P and on the fused prologue (FWD) / epilogue mode as well.
template <int L, int PC, bool FWD>
static RowKernel<float> row_kernel_spec(int mode) {
  if constexpr (FWD) {
    switch (mode) {
      case 0: return k_xfwd_apply<float, 3, L, PC, 0>;
      case 1: return k_xfwd_apply<float, 3, L, PC, 1>;
      case 2: return k_xfwd_apply<float, 3, L, PC, 2>;
      case 4: return k_xfwd_apply<float, 3, L, PC, 4>;
      case 5: return k_xfwd_apply<float, 3, L, PC, 5>;
      default: return nullptr;
    }
  } else {
    switch (mode) {
      case 0: return k_xinv_apply<float, 3, L, PC, 0>;
      case 1: return k_xinv_apply<float, 3, L, PC, 1>;
      case 2: return k_xinv_apply<float, 3, L, PC, 2>;
      case 3: return k_xinv_apply<float, 3, L, PC, 3>;
      case 6: return k_xinv_apply<float, 3, L, PC, 6>;
      default: return nullptr;
    }
  }
}

template <typename T, int M, bool FWD>
static RowKernel<T> row_kernel(int N, int P = 0, int mode = -1) {
  if constexpr (sizeof(T) == 4 && M == 3) {
    if ((P == 1 || P == 2) && mode >= 0) {
      RowKernel<float> k = nullptr;
#define RS(L) k = P == 1 ? row_kernel_spec<L, 1, FWD>(mode) : row_kernel_spec<L, 2, FWD>(mode)
      switch (N) {
        case 48: RS(48); break;
        case 64: RS(64); break;
        case 96: RS(96); break;
        case 128: RS(128); break;
        case 192: RS(192); break;
        case 256: RS(256); break;
        case 384: RS(384); break;
        case 512: RS(512); break;
        case 1024: RS(1024); break;
        default: break;
      }
#undef RS
      if (k) return k;
    }
  }
#define RK(L) return FWD ? k_xfwd_apply<T, M, L, 0, -1> : k_xinv_apply<T, M, L, 0, -1>
  switch (N) {
    case 48: RK(48);
    case 64: RK(64);
    case 96: RK(96);
    case 128: RK(128);
    default: break;
  }
  if constexpr (M == 3) {
    switch (N) {
      case 192: RK(192);
      case 256: RK(256);
      case 384: RK(384);
      case 512: RK(512);
      case 1024: RK(1024);
      default: break;
    }
  }
  RK(0);
#undef RK
}

template <int N, int KC> __global__ void k_col_fused2d(const __grid_constant__ ColGroup<float>);
// variant v = 0, 1, 2 of the fused column pass: 2048 / N >> v columns per block (length
// 1024 has variants 0 and 1 only)
static int fused_variant(int N, int v) { return N >= 1024 && v > 1 ? 1 : v; }
static int fused_cols(int N, int v) { return (2048 / N) >> fused_variant(N, v); }
static ColKernel<float> fused_col_kernel(int N, int v) {
  v = fused_variant(N, v);
#define FK(L) return v == 0 ? k_col_fused2d<L, 2048 / L> : (v == 1 ? k_col_fused2d<L, 1024 / L> : k_col_fused2d<L, 512 / L>)
  switch (N) {
    case 64: FK(64);
    case 128: FK(128);
    case 256: FK(256);
    case 512: FK(512);
    default: return v == 0 ? k_col_fused2d<1024, 2> : k_col_fused2d<1024, 1>;
  }
#undef FK
}
// shared memory of a fused column block: KC columns x 4 channels x N slots
static size_t fused_col_smem(int N, int v) { return (size_t)fused_cols(N, v) * 4 * N * sizeof(float2); }

template <typename T, int M, int MODE>
static ColKernel<T> col_kernel(int N) {
  if constexpr (M == 3 && MODE != 1) return k_col<T, M, MODE, 0>;  // 2D: fused pass only
  switch (N) {
    case 48: return k_col<T, M, MODE, 48>;
    case 64: return k_col<T, M, MODE, 64>;
    case 96: return k_col<T, M, MODE, 96>;
    case 128: return k_col<T, M, MODE, 128>;
    default: break;
  }
  if constexpr (M == 3) {
    switch (N) {
      case 192: return k_col<T, M, MODE, 192>;
      case 256: return k_col<T, M, MODE, 256>;
      case 384: return k_col<T, M, MODE, 384>;
      case 512: return k_col<T, M, MODE, 512>;
      case 1024: return k_col<T, M, MODE, 1024>;
      default: break;
    }
  }
  return k_col<T, M, MODE, 0>;
}
__global__ void k_rot_spec(RotArgs);
template <int M> __global__ void k_grad_spec(SpecOpArgs);
template <int M> __global__ void k_div_spec(SpecOpArgs);
template <int M> __global__ void k_energy_flux(EnergyArgs);
template <int M, typename TK> __global__ void k_energy_w(EnergyArgs, TK *);
__global__ void k_j_contour(JArgs);
template <int M> __global__ void k_xfwd_resid(ResidArgs, FftPlan, int);
template <int M> __global__ void k_xinv_proj(ResidArgs, FftPlan, int, double *);
template <int M, typename TK>
__global__ void k_xinv_resid(ResidArgs, FftPlan, int, TK *, TK *, double *);
template <int M, typename TK> __global__ void k_constitutive(ConstArgs, TK *);
__global__ void k_reduce(const double *, int, int, int, double *);
__global__ void k_reduce_list(ReduceList, double *);
template <typename TK> __global__ void k_kinit(KvArgs<TK>, int, int);
__global__ void k_kfin_init(KrylovScalars *, const double *, int, long long, int, int);
template <typename TK> __global__ void k_kresid(long long, const TK *, const TK *, TK *, double *);
template <typename TK> __global__ void k_norm2(long long, const TK *, double *);
template <typename TK> __global__ void k_maxabs(long long, const TK *, double *);
__global__ void k_kfin_resid(KrylovScalars *, const double *, int, const double *, int);
template <typename TK> __global__ void k_kxr(const __grid_constant__ KvGroup<TK>);
template <typename TK> __global__ void k_kx_finish(const __grid_constant__ KvGroup<TK>);
template <typename TK>
__global__ void k_newton_update(long long, int, const TK *, const TK *, double, double *, double *,
                                const double *, double, double *);
template <typename TA, typename TB> __global__ void k_convert(long long, const TA *, TB *);
template <int M, typename TK> __global__ void k_stag_mask(long long, int, TK *, TK *);
__global__ void k_total_strain(long long, int, const double *, const double *, double, double *);

// ---- error handling --------------------------------------------------------------------
static thread_local char g_err[512] = "";

struct rve;
static void set_err(rve *h, const char *fmt, ...);

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      set_err(h, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return RVE_E_CUDA;                                                              \
    }                                                                                 \
  } while (0)

#define CKL()                                                                         \
  do {                                                                                \
    cudaError_t e_ = cudaGetLastError();                                              \
    if (e_ != cudaSuccess) {                                                          \
      set_err(h, "kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, __LINE__); \
      return RVE_E_CUDA;                                                              \
    }                                                                                 \
  } while (0)

#define TRY(expr)            \
  do {                       \
    int rc_ = (expr);        \
    if (rc_ != RVE_OK) return rc_; \
  } while (0)

// RVE_GRAPHS=0 in the environment disables CUDA-graph replay of the Krylov chunks.
static bool graphs_enabled() {
  const char *e = getenv("RVE_GRAPHS");
  return !(e && e[0] == '0');
}

// ---- the handle ------------------------------------------------------------------------
struct DevPlan {
  FftPlan pf, pd;  // float / double twiddles
};

struct Partials {
  double *cons;   // (m + 1) * Gpw
  double *cmax;   // Gpw
  double *res;    // 5 * Gx
  double *app;    // 6 * Gx (apply: wdp, dots)
  double *kv;     // 2 * Gpw
  double *upd;    // 4 * Gpw
  double *en;     // 2 * Gpw (energy control: dissipated energy, |w|^2)
};

// host state of one BiCGStab solve between chunks
struct KState {
  double bn, rn_best, xE_best, rel;
  bool have_best, finished;
  int restarts, total, st, stall;
};

struct rve {
  rve_desc desc;
  std::string err;
  Geo g;
  int dim, m, c, mixed;
  double t_phase[4];               // host seconds in linearize / E column / Krylov / update (RVE_TIMING)
  int stag_mode;                   // 0 monolithic; 1 / 2: mechanics / phase-field rows only
  double last_e_eps, last_e_phi;   // relative eps / phi change of the last Newton update
  int tr;                          // float32 2D with a compiled column length: transposed
                                   // spectral scratch and the fused column pass
  int n_phases;
  std::vector<uint8_t> phase_host;
  std::vector<double> E_ph, nu_ph, Gc_ph;
  PhaseTab ph;
  double fM[6];
  double C_ref, Lbar, s1;
  cudaStream_t stream;
  // launch geometry
  int Px, Gx, Wy, Wz, Gpw;
  size_t smx_k, smy_k, smz_k, smx_d, smy_d, smz_d;  // dynamic smem (krylov / double)
  int Wy_d, Wz_d, Px_d, Gx_d;
  DevPlan plx, ply, plz;
  // device memory
  uint8_t *mat;
  double *eps_c, *phi_c, *Hn;      // committed
  double *eps_w, *phi_w;           // working (trial) state
  double *sigma, *Hcur, *F, *Lphi, *s2, *fM_d;
  double2 *spec;                   // spectral scratch (float64 sized; float view aliased)
  void *tan;                       // tangent channels (krylov precision)
  void *kv[9];                     // x r rhat p v s t, b (kept rhs), x_best
  KrylovScalars *ks;
  unsigned int *arrive;            // arrival counters of the in-kernel finalisers (x-inverse, k_kxr)
  double *red;                     // reduction outputs (64)
  double *red_h;                   // pinned host mirror
  KrylovScalars *ks_h;             // pinned host mirror
  Partials part;
  double *tabs_d[3][3];            // sn, cs, xi2 per axis (double)
  float *tabs_f[3][3];
  void *tw_d[3], *tw_f[3];
  short *perm[3];                  // digit-reversal tables per axis
  double *ext_dq;                  // scratch for host apply (double, c n + 1)
  double *en;                      // energy control: m n doubles of work space (else NULL)
  // state scalars
  double E_c, tau_c;               // committed
  double E_w;                      // working
  int started;
  int notch_set;
  long long launches;
  // last linearisation
  double lin_gamma, lin_wn, lin_s3, lin_bn2, lin_ref, lin_F3, lin_maxratio;
  double lin_cval;                 // constrained quantity: Gamma, or int G_c gamma_f
  double lin_sigma_sum[6];
  int lin_control;
  double lin_target;
  int lin_valid;
  // newton step bookkeeping
  double step_err;
  double e_scale;                  // column scaling of the E unknown in the current solve
  int tuned;                       // tile schedule chosen by rve_autotune
  int pvar[3];                     // radix plan variant per axis (factorize); 0: compile-time plan
  long long last_applies;          // operator applies of the last increment (batch ordering)
  int own_stream;                  // stream created by the library (destroyed with the handle)
  // host-side fault injection (environment variable RVE_FAULT, read by rve_create):
  // "alloc:<k>" makes the k-th device allocation of rve_create fail as if cudaMalloc had
  // run out of memory; "krylov_breakdown" makes every BiCGStab finaliser of the handle see
  // rho = 0 (a breakdown), which the solver answers with restarts and, after the last one,
  // a failed Newton solve
  int fault_alloc_at, alloc_calls, fault_breakdown;
  // float64 twin of a RVE_MIXED handle (created on first use): an increment whose float32
  // inner solves fail is redone there from the same committed state
  struct rve *twin;
  int fp64_left;   // increments still to run on the float64 twin after a fallback
  cudaStream_t cap_stream;         // private stream for graph capture
  cudaGraphExec_t kgraph;          // one captured chunk of BiCGStab iterations
  int kgraph_launches;             // kernels in the captured chunk
  KState kst;                      // state of the BiCGStab solve in progress
  struct KGroup *kgroup;           // group of a batch call (null when alone)
  bool kdone;                      // group protocol: this member's solve is over
  int krc;                         // group protocol: its status
};

static void set_err(rve *h, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  snprintf(g_err, sizeof g_err, "%s", buf);
  if (h) h->err = buf;
}

// ---- plans and tables --------------------------------------------------------------------
static FDiv host_fdiv(unsigned d) {
  FDiv f;
  f.d = d;
  f.m = d > 1 ? (0xFFFFFFFFu / d) + 1u : 0u;
  return f;
}

// Radix plans of a line length N = 2^a 3^b, stages in DIT order (stage 0 has span 1):
//   variant 0: radix-3 stages, then radix 8 as often as possible, then one 4 or 2 (the plan
//              of the compile-time kernels, stage_plan in fft.cuh);
//   variant 1: the radices of variant 0 in reverse order;
//   variant 2: radix-3 stages, then radix 4 as often as possible, then one 2;
//   variant 3: the radices of variant 2 in reverse order.
// The autotuner picks among them for line lengths that run the runtime-length kernels.
constexpr int kPlanVariants = 4;
static bool factorize(int N, FftPlan &pl, int variant = 0) {
  if (N < 1 || N > 4096) return false;
  int rem = N;
  std::vector<int> R;
  while (rem % 3 == 0) {
    R.push_back(3);
    rem /= 3;
  }
  if (variant < 2) {
    while (rem % 8 == 0) {
      R.push_back(8);
      rem /= 8;
    }
  }
  while (rem % 4 == 0) {
    R.push_back(4);
    rem /= 4;
  }
  while (rem % 2 == 0) {
    R.push_back(2);
    rem /= 2;
  }
  if (rem != 1) return false;
  if (variant == 1 || variant == 3) std::reverse(R.begin(), R.end());
  if (R.empty()) R.push_back(1);  // N = 1: a single trivial stage
  if ((int)R.size() > FFT_MAX_STAGES) return false;
  memset(&pl, 0, sizeof pl);
  pl.N = N;
  pl.Np = N + (N - 1) / 8;
  pl.S = (int)R.size();
  int ns = 1;
  for (int s = 0; s < pl.S; ++s) {
    pl.R[s] = R[s];
    pl.Ns[s] = ns;
    pl.dNs[s] = host_fdiv((unsigned)ns);
    pl.dNb[s] = host_fdiv((unsigned)(N / R[s]));
    ns *= R[s];
  }
  return true;
}

// digit reversal (position -> DIT input sample index) of a plan, see fft.cuh
static int host_digit_reverse(const FftPlan &pl, int p) {
  int out = 0, mul = 1, len = pl.N;
  for (int s = pl.S - 1; s >= 0; --s) {
    const int R = pl.R[s];
    len /= R;
    const int r = p / len;
    p -= r * len;
    out += r * mul;
    mul *= R;
  }
  return out;
}

static int make_plan(rve *h, int N, DevPlan &dp, void **twd, void **twf, short **perm) {
  FftPlan pl;
  if (!factorize(N, pl)) {
    set_err(h, "grid extent %d is not of the form 2^a 3^b <= 4096", N);
    return RVE_E_ARG;
  }
  std::vector<double2> td(N);
  std::vector<float2> tf(N);
  for (int k = 0; k < N; ++k) {
    const double a = 2.0 * M_PI * (double)k / (double)N;
    td[k] = make_double2(cos(a), -sin(a));
    tf[k] = make_float2((float)td[k].x, (float)td[k].y);
  }
  std::vector<short> pr(2 * N);
  for (int p = 0; p < N; ++p) {
    const int r = host_digit_reverse(pl, p);
    pr[p] = (short)r;        // rev: position -> index
    pr[N + r] = (short)p;    // unrev: index -> position
  }
  CK(cudaMallocAsync(twd, sizeof(double2) * N, 0));
  CK(cudaMallocAsync(twf, sizeof(float2) * N, 0));
  CK(cudaMallocAsync((void **)perm, sizeof(short) * 2 * N, 0));
  CK(cudaMemcpy(*twd, td.data(), sizeof(double2) * N, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(*twf, tf.data(), sizeof(float2) * N, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(*perm, pr.data(), sizeof(short) * 2 * N, cudaMemcpyHostToDevice));
  pl.rev = *perm;
  pl.unrev = *perm + N;
  dp.pd = pl;
  dp.pd.tw = *twd;
  dp.pf = pl;
  dp.pf.tw = *twf;
  return RVE_OK;
}

// Replace axis a's radix plan by variant v: the same twiddle tables, a new stage list and new
// digit-reversal tables (rebuilt here and copied over the axis's table).  Chunk graphs
// captured with the old plan are dropped.
static int set_plan_variant(rve *h, int a, int v) {
  const int N = a == 0 ? h->g.nx : (a == 1 ? h->g.ny : h->g.nz);
  FftPlan pl;
  if (!factorize(N, pl, v)) {
    set_err(h, "no radix plan variant %d for length %d", v, N);
    return RVE_E_ARG;
  }
  std::vector<short> pr(2 * N);
  for (int p = 0; p < N; ++p) {
    const int r = host_digit_reverse(pl, p);
    pr[p] = (short)r;
    pr[N + r] = (short)p;
  }
  CK(cudaStreamSynchronize(h->stream));  // nothing of the handle reads the table meanwhile
  CK(cudaMemcpy(h->perm[a], pr.data(), sizeof(short) * 2 * N, cudaMemcpyHostToDevice));
  DevPlan &dp = a == 0 ? h->plx : (a == 1 ? h->ply : h->plz);
  const void *twd = dp.pd.tw, *twf = dp.pf.tw;
  pl.rev = h->perm[a];
  pl.unrev = h->perm[a] + N;
  dp.pd = pl;
  dp.pd.tw = twd;
  dp.pf = pl;
  dp.pf.tw = twf;
  h->pvar[a] = v;
  if (h->kgraph) {
    cudaGraphExecDestroy(h->kgraph);
    h->kgraph = nullptr;
  }
  return RVE_OK;
}

// Line length that selects the pass kernels of axis a: the length itself (its compile-time
// kernel, where one is built) under plan variant 0, else 0 (the runtime-length kernel, which
// reads the stage list from the plan).
static int ct_len(const rve *h, int a) {
  const int N = a == 0 ? h->g.nx : (a == 1 ? h->g.ny : h->g.nz);
  return h->pvar[a] == 0 ? N : 0;
}

// lengths with compile-time pass kernels (kernels_fft_<N>.cu): 2D all nine, 3D up to 128
static bool has_ct_kernel(int N, int m) {
  static const int ct[9] = {48, 64, 96, 128, 192, 256, 384, 512, 1024};
  const int cnt = m == 3 ? 9 : 4;
  for (int i = 0; i < cnt; ++i)
    if (ct[i] == N) return true;
  return false;
}

// variants of N whose stage lists differ from every lower variant's
static std::vector<int> distinct_variants(int N) {
  std::vector<int> out;
  std::vector<std::vector<int>> seen;
  for (int v = 0; v < kPlanVariants; ++v) {
    FftPlan pl;
    if (!factorize(N, pl, v)) continue;
    std::vector<int> rs(pl.R, pl.R + pl.S);
    bool dup = false;
    for (auto &q : seen) dup = dup || q == rs;
    if (dup) continue;
    seen.push_back(rs);
    out.push_back(v);
  }
  return out;
}

// RVE_RADIX_PLAN=<v> in the environment fixes plan variant v (where it differs from variant 0)
// on every axis except the column axis of the fused 2D pass, compile-time lengths included
// (they then run the runtime-length kernels), and turns off the tuner's plan choice.
static int forced_plan_variant() {
  const char *e = getenv("RVE_RADIX_PLAN");
  if (!e) return -1;
  const int v = atoi(e);
  return v >= 0 && v < kPlanVariants ? v : -1;
}

// Per-axis tables of the projection direction and |xi|^2.  The direction along axis a is
// n_a ~ sn_a(k_a) prod_{b != a} cs_b(k_b): rotated scheme sn = sin(q/2), cs = cos(q/2)
// (exactly 0 at the Nyquist index); continuous frequencies sn = xi (0 at the Nyquist
// index), cs = 1.
static int make_axis_tables(rve *h, int a, int N, int gamma_op) {
  std::vector<double> sn(N), cs(N), x2(N);
  for (int k = 0; k < N; ++k) {
    int ks = (2 * k < N) ? k : k - N;  // Nyquist (2k == N) -> -N/2
    const double q = M_PI * (double)ks / (double)N;
    const double xi = 2.0 * M_PI * (double)ks / (double)N;
    if (gamma_op == RVE_GAMMA_CONTINUOUS) {
      sn[k] = (2 * k == N) ? 0.0 : xi;
      cs[k] = 1.0;
    } else {
      sn[k] = sin(q);
      cs[k] = (2 * k == N) ? 0.0 : cos(q);
    }
    x2[k] = xi * xi;
  }
  const std::vector<double> *src[3] = {&sn, &cs, &x2};
  for (int t = 0; t < 3; ++t) {
    CK(cudaMallocAsync((void **)&h->tabs_d[a][t], sizeof(double) * N, 0));
    CK(cudaMallocAsync((void **)&h->tabs_f[a][t], sizeof(float) * N, 0));
    std::vector<float> f(N);
    for (int k = 0; k < N; ++k) f[k] = (float)(*src[t])[k];
    CK(cudaMemcpy(h->tabs_d[a][t], src[t]->data(), sizeof(double) * N, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->tabs_f[a][t], f.data(), sizeof(float) * N, cudaMemcpyHostToDevice));
  }
  return RVE_OK;
}

static size_t pow2_floor(size_t x) {
  size_t p = 1;
  while (p * 2 <= x) p *= 2;
  return p;
}

static int padded(int N) { return N + (N - 1) / 8; }

// launch geometry of the FFT passes for element size es (bytes of one real value):
// P row pairs per x-pass block, W kx columns per column-pass block.  P and W come from the
// tuner (rve_tune) or these defaults.
static void pass_geometry(const Geo &g, int es, int Preq, int Wreq, int &P, int &Gx, int &Wy, int &Wz,
                          size_t &smx, size_t &smy, size_t &smz) {
  const size_t budget = 120 * 1024;
  const int npx = padded(g.nx);
  P = Preq > 0 ? Preq : (int)(1024 / g.nx);
  if (P < 1) P = 1;
  while (P > 1 && (size_t)g.c * P * npx * 2 * es > budget) P /= 2;
  if (2 * P > g.rows + 1) P = (g.rows + 1) / 2;
  if (P < 1) P = 1;
  Gx = (g.rows + 2 * P - 1) / (2 * P);
  smx = (size_t)g.c * P * npx * 2 * es;
  auto colW = [&](int N) {
    size_t per = (size_t)g.c * padded(N) * 2 * es;  // one column, all channels, complex
    size_t w = Wreq > 0 ? (size_t)Wreq : budget / per;
    if (w < 1) w = 1;
    w = pow2_floor(w);
    if (w > 16) w = 16;
    while (w > 1 && per * w > budget) w /= 2;
    while (w > 1 && w / 2 >= (size_t)g.hx) w /= 2;
    return (int)w;
  };
  Wy = colW(g.ny);
  Wz = g.nz > 1 ? colW(g.nz) : 1;
  smy = (size_t)g.c * padded(g.ny) * Wy * 2 * es;
  smz = (size_t)g.c * padded(g.nz) * Wz * 2 * es;
}

// Opt every FFT-pass kernel in to the largest dynamic shared memory the device allows
// (the opt-in per-block limit minus the kernel's own static shared memory).
static int set_one_attr(rve *h, const void *k, int optin) {
  cudaFuncAttributes fa;
  CK(cudaFuncGetAttributes(&fa, k));
  const int mx = optin - (int)fa.sharedSizeBytes;
  CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  return RVE_OK;
}

static int set_smem_attrs(rve *h, size_t need) {
  static int done_dev = -1;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  int optin = 0;
  CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if ((size_t)optin < need + 4096) {
    set_err(h, "FFT pass needs %zu bytes of shared memory; the device allows %d", need, optin);
    return RVE_E_ARG;
  }
  if (done_dev == dev) return RVE_OK;
#define SA(...) TRY(set_one_attr(h, (const void *)(__VA_ARGS__), optin))
  static const int kAllCt[9] = {48, 64, 96, 128, 192, 256, 384, 512, 1024};  // kernels_fft_<N>.cu
  for (int li = -1; li < 9; ++li) {
    const int N = li < 0 ? 0 : kAllCt[li];
    const bool pow2 = (N & (N - 1)) == 0;
    SA((row_kernel<float, 3, true>(N))); SA((row_kernel<float, 3, false>(N)));
    for (int pc = 1; pc <= 2 && N > 0; ++pc)
      for (int md = 0; md <= 6; ++md) {
        if (md != 3 && md != 6) SA((row_kernel<float, 3, true>(N, pc, md)));
        if (md != 4 && md != 5) SA((row_kernel<float, 3, false>(N, pc, md)));
      }
    SA((row_kernel<float, 6, true>(N))); SA((row_kernel<float, 6, false>(N)));
    SA((row_kernel<double, 3, true>(N))); SA((row_kernel<double, 3, false>(N)));
    SA((row_kernel<double, 6, true>(N))); SA((row_kernel<double, 6, false>(N)));
    SA((col_kernel<float, 3, 1>(N))); SA((col_kernel<double, 3, 1>(N)));
    SA((col_kernel<float, 6, 0>(N))); SA((col_kernel<float, 6, 1>(N))); SA((col_kernel<float, 6, 2>(N)));
    SA((col_kernel<double, 6, 0>(N))); SA((col_kernel<double, 6, 1>(N))); SA((col_kernel<double, 6, 2>(N)));
    if (N > 0 && pow2)
      for (int v = 0; v < 3; ++v) SA(fused_col_kernel(N, v));
  }
  SA((col_kernel<double, 3, 0>(0))); SA((col_kernel<double, 3, 2>(0)));  // J-integral rotation
  SA(k_xfwd_resid<3>); SA(k_xfwd_resid<6>);
  SA(k_xinv_proj<3>); SA(k_xinv_proj<6>);
  SA((k_xinv_resid<3, float>)); SA((k_xinv_resid<6, float>));
  SA((k_xinv_resid<3, double>)); SA((k_xinv_resid<6, double>));
#undef SA
  done_dev = dev;
  return RVE_OK;
}

// ---- typed launch helpers ----------------------------------------------------------------
template <typename T> static const DevPlan *plans_of(const rve *h, int a) {
  return a == 0 ? &h->plx : (a == 1 ? &h->ply : &h->plz);
}
template <typename T> static FftPlan plan_of(const rve *h, int a);
template <> FftPlan plan_of<float>(const rve *h, int a) { return plans_of<float>(h, a)->pf; }
template <> FftPlan plan_of<double>(const rve *h, int a) { return plans_of<double>(h, a)->pd; }
template <typename T> static AxisTab<T> tabs_of(const rve *h);
template <> AxisTab<float> tabs_of<float>(const rve *h) {
  AxisTab<float> t;
  for (int a = 0; a < 3; ++a) {
    t.sn[a] = h->tabs_f[a][0];
    t.cs[a] = h->tabs_f[a][1];
    t.xi2[a] = h->tabs_f[a][2];
  }
  return t;
}
template <> AxisTab<double> tabs_of<double>(const rve *h) {
  AxisTab<double> t;
  for (int a = 0; a < 3; ++a) {
    t.sn[a] = h->tabs_d[a][0];
    t.cs[a] = h->tabs_d[a][1];
    t.xi2[a] = h->tabs_d[a][2];
  }
  return t;
}

// transposed spectral scratch + fused column pass for this precision and dimension
template <typename T, int M>
static int spec_tr(const rve *h) {
  return (sizeof(T) == 4 && M == 3 && h->tr) ? 1 : 0;
}

// column passes (after the x-forward pass, before the x-inverse pass) for precision T, over
// nm RVEs of h's shape (scratch spec[i], Krylov scalars ks[i]) as one launch per pass
template <typename T, int M>
static int launch_columns_n(rve *h, cpx<T> *const *spec, const KrylovScalars *const *ks, int nm, int Wy,
                            int Wz, size_t smy, size_t smz, cudaStream_t st) {
  ColGroup<T> G;
  memset((void *)&G, 0, sizeof G);
  ColArgs<T> &ca = G.base;
  ca.g = h->g;
  ca.spec = spec[0];
  ca.tab = tabs_of<T>(h);
  ca.inv_n = (T)(1.0 / (double)h->g.n);
  ca.ks = ks[0];
  ca.yplan = plan_of<T>(h, 1);
  for (int i = 0; i < nm; ++i) {
    G.spec[i] = spec[i];
    G.ks[i] = ks[i];
  }
  const Geo &g = h->g;
  auto log2i = [](int w) {
    int l = 0;
    while ((1 << l) < w) ++l;
    return l;
  };
  if (spec_tr<T, M>(h)) {
    ca.axis = 1;
    ca.W = 1;
    ca.lw = 0;
    ca.plan = plan_of<T>(h, 1);
    // the column tile Wy of the tuner selects the variant: 1 -> 2048 / N columns per block,
    // 2 -> half, 4 and more -> a quarter
    const int v = Wy >= 4 ? 2 : (Wy >= 2 ? 1 : 0);
    const int kc = fused_cols(g.ny, v);
    dim3 grid((g.hx + kc - 1) / kc, nm);
    fused_col_kernel(g.ny, v)<<<grid, kc * g.ny / 2, fused_col_smem(g.ny, v), st>>>(
        *reinterpret_cast<ColGroup<float> *>(&G));
    h->launches += 1;
  } else if (g.nz == 1) {
    ca.axis = 1;
    ca.W = Wy;
    ca.lw = log2i(Wy);
    ca.plan = plan_of<T>(h, 1);
    dim3 grid((g.hx + Wy - 1) / Wy, 1, nm);
    col_kernel<T, M, 1>(ct_len(h, 1))<<<grid, 256, smy, st>>>(G);
    h->launches += 1;
  } else {
    ca.axis = 1;
    ca.W = Wy;
    ca.lw = log2i(Wy);
    ca.plan = plan_of<T>(h, 1);
    dim3 gy((g.hx + Wy - 1) / Wy, g.nz, nm);
    col_kernel<T, M, 0>(ct_len(h, 1))<<<gy, 256, smy, st>>>(G);
    ca.axis = 2;
    ca.W = Wz;
    ca.lw = log2i(Wz);
    ca.plan = plan_of<T>(h, 2);
    dim3 gz((g.hx + Wz - 1) / Wz, g.ny, nm);
    col_kernel<T, M, 1>(ct_len(h, 2))<<<gz, 256, smz, st>>>(G);
    ca.axis = 1;
    ca.W = Wy;
    ca.lw = log2i(Wy);
    ca.plan = plan_of<T>(h, 1);
    col_kernel<T, M, 2>(ct_len(h, 1))<<<gy, 256, smy, st>>>(G);
    h->launches += 3;
  }
  CKL();
  return RVE_OK;
}

template <typename T, int M>
static int launch_columns(rve *h, cpx<T> *spec, const KrylovScalars *ks, int Wy, int Wz, size_t smy,
                          size_t smz) {
  return launch_columns_n<T, M>(h, &spec, &ks, 1, Wy, Wz, smy, smz, h->stream);
}

// ---- the scaled operator apply y = S J x ------------------------------------------------
template <typename TK, int M>
static ApplyArgs<TK> apply_args(rve *h, TK *x, const double *xE_ptr, TK *y, int pro_mode, int epi_mode,
                                const TK *r, const TK *v, const TK *rhat, const TK *s, const KrylovScalars *ks) {
  ApplyArgs<TK> a;
  memset((void *)&a, 0, sizeof a);
  a.g = h->g;
  a.x = x;
  a.y = y;
  a.tan = (const TK *)h->tan;
  a.xE_ptr = xE_ptr;
  a.e_scale = (ks != nullptr) ? h->e_scale : 1.0;
  for (int k = 0; k < 6; ++k) a.fM[k] = h->fM[k];
  a.spec = (cpx<TK> *)h->spec;
  a.part = h->part.app;
  a.pro_mode = pro_mode;
  a.r = const_cast<TK *>(r);  // written by prologue mode 5 only
  a.v = v;
  a.rhat = rhat;
  a.s = s;
  a.epi_mode = epi_mode;
  a.ks = ks;
  a.tr = spec_tr<TK, M>(h);
  return a;
}

// spec / part: spectral scratch and reduction partials of the passes (null: the handle's own)
template <typename TK, int M>
static int apply_scaled(rve *h, TK *x, const double *xE_ptr, TK *y, int pro_mode, int epi_mode,
                        const TK *r, const TK *v, const TK *rhat, const TK *s, const KrylovScalars *ks,
                        cpx<TK> *spec = nullptr, double *part = nullptr, double *yE = nullptr) {
  ApplyArgs<TK> a;
  memset((void *)&a, 0, sizeof a);
  a.g = h->g;
  a.x = x;
  a.y = y;
  a.tan = (const TK *)h->tan;
  a.xE_ptr = xE_ptr;
  a.e_scale = (ks != nullptr) ? h->e_scale : 1.0;
  for (int k = 0; k < 6; ++k) a.fM[k] = h->fM[k];
  a.spec = spec ? spec : (cpx<TK> *)h->spec;
  a.part = part ? part : h->part.app;
  if (yE) {  // the x-inverse pass also writes the E slot of y (no separate reduction launch)
    a.fin = h->lin_control == RVE_CTRL_STRAIN ? 4 : 3;
    a.yE = yE;
  }
  a.pro_mode = pro_mode;
  a.r = const_cast<TK *>(r);  // written by prologue mode 5 only
  a.v = v;
  a.rhat = rhat;
  a.s = s;
  a.epi_mode = epi_mode;
  a.ks = ks;
  a.tr = spec_tr<TK, M>(h);
  const bool dbl = sizeof(TK) == 8;
  const int P = dbl ? h->Px_d : h->Px;
  const int Gx = dbl ? h->Gx_d : h->Gx;
  const size_t smx = dbl ? h->smx_d : h->smx_k;
  row_kernel<TK, M, true>(ct_len(h, 0), P, a.pro_mode)<<<Gx, 256, smx, h->stream>>>(solo(a), plan_of<TK>(h, 0), P);
  h->launches += 1;
  CKL();
  TRY((launch_columns<TK, M>(h, a.spec, ks, dbl ? h->Wy_d : h->Wy, dbl ? h->Wz_d : h->Wz,
                             dbl ? h->smy_d : h->smy_k, dbl ? h->smz_d : h->smz_k)));
  row_kernel<TK, M, false>(ct_len(h, 0), P, a.epi_mode)<<<Gx, 256, smx, h->stream>>>(solo(a), plan_of<TK>(h, 0), P);
  h->launches += 1;
  CKL();
  return RVE_OK;
}

// ---- host <- device reductions -----------------------------------------------------------
static int reduce_to_host(rve *h, const double *part, int G, int NQ, int is_max, double *out) {
  k_reduce<<<1, 256, 0, h->stream>>>(part, G, NQ, is_max, h->red);
  h->launches += 1;
  CKL();
  CK(cudaMemcpyAsync(h->red_h, h->red, sizeof(double) * NQ, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int q = 0; q < NQ; ++q) out[q] = h->red_h[q];
  return RVE_OK;
}

// the segments of L in one launch and one copy (same per-quantity arithmetic as
// reduce_to_host); out receives the quantities of all segments in order
static int reduce_list_to_host(rve *h, ReduceList L, double *out) {
  int tot = 0;
  for (int i = 0; i < L.n; ++i) {
    L.s[i].off = tot;
    tot += L.s[i].NQ;
  }
  k_reduce_list<<<1, 256, 0, h->stream>>>(L, h->red);
  h->launches += 1;
  CKL();
  CK(cudaMemcpyAsync(h->red_h, h->red, sizeof(double) * tot, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int q = 0; q < tot; ++q) out[q] = h->red_h[q];
  return RVE_OK;
}

// ---- energy-controlled constraint (Eq. SystemDisc) ---------------------------------------
// Column passes of the float64 residual layout without a spectral operator in between:
// forward (DIF, positions stay digit-reversed) or inverse (DIT).
template <int M>
static int spec_columns(rve *h, cpx<double> *spec, bool forward) {
  const Geo &g = h->g;
  ColGroup<double> G;
  memset((void *)&G, 0, sizeof G);
  ColArgs<double> &ca = G.base;
  ca.g = g;
  ca.spec = spec;
  ca.tab = tabs_of<double>(h);
  ca.inv_n = 1.0 / (double)g.n;
  ca.yplan = plan_of<double>(h, 1);
  G.spec[0] = spec;
  auto log2i = [](int w) {
    int l = 0;
    while ((1 << l) < w) ++l;
    return l;
  };
  auto pass = [&](int axis, bool fwd) {
    ca.axis = axis;
    ca.W = axis == 1 ? h->Wy_d : h->Wz_d;
    ca.lw = log2i(ca.W);
    ca.plan = plan_of<double>(h, axis);
    const dim3 grid((g.hx + ca.W - 1) / ca.W, axis == 1 ? g.nz : g.ny, 1);
    const size_t sm = axis == 1 ? h->smy_d : h->smz_d;
    if (fwd) col_kernel<double, M, 0>(ct_len(h, axis))<<<grid, 256, sm, h->stream>>>(G);
    else col_kernel<double, M, 2>(ct_len(h, axis))<<<grid, 256, sm, h->stream>>>(G);
    h->launches += 1;
  };
  if (forward) {
    pass(1, true);
    if (g.nz > 1) pass(2, true);
  } else {
    if (g.nz > 1) pass(2, false);
    pass(1, false);
  }
  CKL();
  return RVE_OK;
}

// D = sum_v G_c (phi^2 / (2 l) + (l / 2) sum_a (D_a phi)^2) and w = dD/dphi = G_c phi / l +
// l sum_a D_a^T (G_c D_a phi) (0 on the notch) into the constraint-row tangent channel, with
// the spectral derivative D_a of Eq. newGammaFourier: two float64 FFT round trips through
// the residual layout.  Leaves the partials of D and |w|^2 in part.en.
template <typename TK, int M>
static int energy_constraint_t(rve *h, const double *phi) {
  const Geo &g = h->g;
  ResidArgs ra;
  memset(&ra, 0, sizeof ra);
  ra.g = g;
  ra.sigma = h->en;  // transformed alongside phi; only channel m (phi) is read
  ra.phi = phi;
  ra.spec = (cpx<double> *)h->spec;
  SpecOpArgs so;
  so.g = g;
  so.spec = ra.spec;
  so.yrev = plan_of<double>(h, 1).rev;
  so.zrev = plan_of<double>(h, 2).rev;
  so.inv_n = 1.0 / (double)g.n;
  EnergyArgs ea;
  ea.g = g;
  ea.phi = phi;
  ea.mat = h->mat;
  ea.ph = h->ph;
  ea.ell = h->desc.ell;
  ea.buf = h->en;
  ea.part = h->part.en;
  // gradient D_a phi -> en[a]
  k_xfwd_resid<M><<<h->Gx_d, 256, h->smx_d, h->stream>>>(ra, plan_of<double>(h, 0), h->Px_d);
  CKL();
  TRY(spec_columns<M>(h, ra.spec, true));
  k_grad_spec<M><<<h->Gpw, 256, 0, h->stream>>>(so);
  CKL();
  TRY(spec_columns<M>(h, ra.spec, false));
  k_xinv_proj<M><<<h->Gx_d, 256, h->smx_d, h->stream>>>(ra, plan_of<double>(h, 0), h->Px_d, h->en);
  CKL();
  // flux G_c D_a phi (in place) and the dissipated energy
  k_energy_flux<M><<<h->Gpw, 256, 0, h->stream>>>(ea);
  CKL();
  // sum_a D_a^T flux_a -> en[0]
  k_xfwd_resid<M><<<h->Gx_d, 256, h->smx_d, h->stream>>>(ra, plan_of<double>(h, 0), h->Px_d);
  CKL();
  TRY(spec_columns<M>(h, ra.spec, true));
  k_div_spec<M><<<h->Gpw, 256, 0, h->stream>>>(so);
  CKL();
  TRY(spec_columns<M>(h, ra.spec, false));
  k_xinv_proj<M><<<h->Gx_d, 256, h->smx_d, h->stream>>>(ra, plan_of<double>(h, 0), h->Px_d, h->en);
  CKL();
  k_energy_w<M, TK><<<h->Gpw, 256, 0, h->stream>>>(ea, (TK *)h->tan);
  CKL();
  h->launches += 8;
  return RVE_OK;
}

// ---- linearisation: constitutive law + residual + rhs ------------------------------------
template <typename TK, int M>
static int linearize_t(rve *h, const double *eps_t, const double *phi, double E, int control,
                       double target) {
  const Geo &g = h->g;
  ConstArgs ca;
  ca.g = g;
  ca.eps_t = eps_t;
  ca.phi = phi;
  ca.Hn = h->Hn;
  ca.mat = h->mat;
  ca.ph = h->ph;
  for (int k = 0; k < 6; ++k) ca.fM[k] = h->fM[k];
  ca.E = E;
  ca.ell = h->desc.ell;
  ca.k_res = h->desc.k_res;
  ca.s1 = h->s1;
  ca.Lbar = h->Lbar;
  ca.isotropic = h->desc.split == RVE_SPLIT_NONE;
  ca.sigma = h->sigma;
  ca.H = h->Hcur;
  ca.part = h->part.cons;
  ca.part_max = h->part.cmax;
  k_constitutive<M, TK><<<h->Gpw, 256, 0, h->stream>>>(ca, (TK *)h->tan);
  h->launches += 1;
  CKL();
  ResidArgs ra;
  ra.g = g;
  ra.sigma = h->sigma;
  ra.phi = phi;
  ra.H = h->Hcur;
  ra.mat = h->mat;
  ra.ph = h->ph;
  ra.ell = h->desc.ell;
  ra.s1 = h->s1;
  ra.Lbar = h->Lbar;
  ra.spec = (cpx<double> *)h->spec;
  ra.F = h->F;
  ra.Lphi = h->Lphi;
  ra.part = h->part.res;
  k_xfwd_resid<M><<<h->Gx_d, 256, h->smx_d, h->stream>>>(ra, plan_of<double>(h, 0), h->Px_d);
  h->launches += 1;
  CKL();
  TRY((launch_columns<double, M>(h, ra.spec, nullptr, h->Wy_d, h->Wz_d, h->smy_d, h->smz_d)));
  TK *rvec = (TK *)h->kv[1];
  k_xinv_resid<M, TK><<<h->Gx_d, 256, h->smx_d, h->stream>>>(ra, plan_of<double>(h, 0), h->Px_d,
                                                             rvec, (TK *)h->tan, h->s2);
  h->launches += 1;
  CKL();
  const bool energy = h->desc.constraint == RVE_CONSTRAINT_ENERGY;
  if (energy) TRY((energy_constraint_t<TK, M>(h, phi)));
  if (h->stag_mode) {
    k_stag_mask<M, TK><<<h->Gpw, 256, 0, h->stream>>>(g.n, h->stag_mode, (TK *)h->tan, rvec);
    h->launches += 1;
    CKL();
  }
  double cs[8], cm[1], rs[5], red[M + 7];
  {
    ReduceList L;
    memset(&L, 0, sizeof L);
    L.s[0] = {h->part.cons, h->Gpw, M + 1, 0, 0};
    L.s[1] = {h->part.cmax, h->Gpw, 1, 1, 0};
    L.s[2] = {h->part.res, h->Gx_d, 5, 0, 0};
    L.n = 3;
    TRY(reduce_list_to_host(h, L, red));
    for (int q = 0; q <= M; ++q) cs[q] = red[q];
    cm[0] = red[M + 1];
    for (int q = 0; q < 5; ++q) rs[q] = red[M + 2 + q];
  }
  for (int k = 0; k < M; ++k) h->lin_sigma_sum[k] = cs[k];
  const double ref2 = cs[M] + rs[4];
  h->lin_maxratio = cm[0];
  h->lin_gamma = rs[0];
  h->lin_wn = sqrt(rs[1]);
  h->lin_cval = h->lin_gamma;
  if (energy) {
    double es[2];
    TRY(reduce_to_host(h, h->part.en, h->Gpw, 2, 0, es));
    h->lin_cval = es[0];
    h->lin_wn = sqrt(es[1]);
  }
  double s3, F3, gref;
  if (control == RVE_CTRL_CRACK) {
    s3 = h->lin_wn > 0 ? 1.0 / h->lin_wn : 1.0;
    F3 = h->lin_cval - target;
    gref = s3 * fmax(fabs(h->lin_cval), fabs(target));
  } else {
    s3 = 1.0;
    F3 = E - target;
    gref = fmax(fabs(E), fabs(target));
  }
  h->lin_s3 = s3;
  h->lin_F3 = F3;
  const double bE = -s3 * F3;
  // |b|^2 of the rows in the solve (staggered sub-solves keep one block of rows)
  h->lin_bn2 = (h->stag_mode == 2 ? 0.0 : rs[2]) + (h->stag_mode == 1 ? 0.0 : rs[3]) + bE * bE;
  h->lin_ref = sqrt(ref2 + gref * gref);
  h->lin_control = control;
  h->lin_target = target;
  h->lin_valid = 1;
  // Krylov scalars of the coming solve
  KrylovScalars *k = h->ks_h;
  memset(k, 0, sizeof *k);
  k->rE = bE;
  k->bE = bE;
  k->bn2 = h->lin_bn2;
  k->rn2 = h->lin_bn2;
  k->s3 = s3;
  k->strain = control == RVE_CTRL_STRAIN ? 1 : 0;
  k->escale = 1.0;
  const double kt = h->desc.krylov_tol;
  k->tol2 = kt * kt;
  const double atol = 0.1 * 1e-13 * h->lin_ref;
  k->atol2 = atol * atol;
  k->maxit = h->desc.krylov_max;
  k->fault_rho0 = h->fault_breakdown;
  CK(cudaMemcpyAsync(h->ks, k, sizeof *k, cudaMemcpyHostToDevice, h->stream));
  return RVE_OK;
}

static int linearize(rve *h, const double *eps_t, const double *phi, double E, int control,
                     double target) {
  if (h->mixed) {
    if (h->m == 3) return linearize_t<float, 3>(h, eps_t, phi, E, control, target);
    return linearize_t<float, 6>(h, eps_t, phi, E, control, target);
  }
  if (h->m == 3) return linearize_t<double, 3>(h, eps_t, phi, E, control, target);
  return linearize_t<double, 6>(h, eps_t, phi, E, control, target);
}

// ---- BiCGStab on the device --------------------------------------------------------------
// BiCGStab with restarts (same rule as the oracle): every chunk of iterations the host
// reads the device scalars; the iterate with the smallest residual is kept; on breakdown,
// a non-finite residual or a 1e6-fold growth over the best, the solve restarts from the
// kept iterate (r = b - A x) with the next shadow seed, at most kMaxRestarts times.
static int krylov_chunk_len() {
  static const int k = [] {
    const char *e = getenv("RVE_KCHUNK");
    const int v = e ? atoi(e) : 0;
    return v > 0 && v <= 64 ? v : 8;
  }();
  return k;
}

template <typename TK>
static KvArgs<TK> kv_args(rve *h) {
  KvArgs<TK> kv;
  kv.len = (long long)h->c * h->g.n;
  kv.c = h->c;
  kv.n = h->g.n;
  kv.x = (TK *)h->kv[0];
  kv.r = (TK *)h->kv[1];
  kv.rhat = (TK *)h->kv[2];
  kv.p = (TK *)h->kv[3];
  kv.v = (TK *)h->kv[4];
  kv.s = (TK *)h->kv[5];
  kv.t = (TK *)h->kv[6];
  kv.ks = h->ks;
  kv.part = h->part.kv;
  kv.G = h->Gpw;
  kv.arrive = nullptr;
  return kv;
}

// start of a solve: keep b, shadow vector, rho; on the handle's stream
template <typename TK, int M>
static int kry_begin(rve *h) {
  KState &S = h->kst;
  KvArgs<TK> kv = kv_args<TK>(h);
  TK *bsave = (TK *)h->kv[7];
  const size_t vbytes = sizeof(TK) * (size_t)kv.len;
  CK(cudaMemcpyAsync(bsave, kv.r, vbytes, cudaMemcpyDeviceToDevice, h->stream));
  k_kinit<TK><<<h->Gpw, 256, 0, h->stream>>>(kv, 0, 1);
  k_kfin_init<<<1, 256, 0, h->stream>>>(h->ks, h->part.kv, h->Gpw, kv.len, 0, 1);
  h->launches += 2;
  CKL();
  S.bn = sqrt(h->lin_bn2);
  S.rn_best = S.bn;
  S.xE_best = 0.0;
  S.have_best = false;
  S.restarts = 0;
  S.total = 0;
  S.st = 1;
  S.stall = 0;
  S.rel = 1.0;
  S.finished = false;
  return RVE_OK;
}

// after a chunk, with the device scalars copied to h->ks_h: convergence, best iterate,
// restarts (issued on h->stream); sets kst.finished when the solve is over
template <typename TK, int M>
static int kry_after_chunk(rve *h) {
  const int kMaxRestarts = 6, kStallChecks = 25;
  KState &S = h->kst;
  KvArgs<TK> kv = kv_args<TK>(h);
  TK *bsave = (TK *)h->kv[7], *xbest = (TK *)h->kv[8];
  const size_t vbytes = sizeof(TK) * (size_t)kv.len;
  const int Gx = sizeof(TK) == 8 ? h->Gx_d : h->Gx;
  const KrylovScalars &k = *h->ks_h;
  S.total = k.iters;
  const double rn = sqrt(k.rn2);
  if (k.done && k.status == 0) {
    S.st = 0;
    S.rel = S.bn > 0 ? rn / S.bn : 0.0;
    S.finished = true;
    return RVE_OK;
  }
  if (k.done && k.status == 1) {  // iteration limit: the better of the last and the kept iterate
    S.st = 1;
    S.rel = S.bn > 0 ? rn / S.bn : 0.0;
    if (S.have_best && !(rn < S.rn_best)) {
      CK(cudaMemcpyAsync(kv.x, xbest, vbytes, cudaMemcpyDeviceToDevice, h->stream));
      h->ks_h->xE = S.xE_best;
      S.rel = S.bn > 0 ? S.rn_best / S.bn : 0.0;
    }
    S.finished = true;
    return RVE_OK;
  }
  bool bad = (k.done && k.status == 2) || !isfinite(rn) || rn > 1e6 * S.rn_best;
  if (!bad) {
    if (rn < S.rn_best) {
      S.rn_best = rn;
      S.xE_best = k.xE;
      S.have_best = true;
      S.stall = 0;
      CK(cudaMemcpyAsync(xbest, kv.x, vbytes, cudaMemcpyDeviceToDevice, h->stream));
      return RVE_OK;
    }
    if (++S.stall < kStallChecks) return RVE_OK;
    S.stall = 0;
    bad = true;
  }
  if (S.restarts >= kMaxRestarts) {
    S.st = 2;
    S.finished = true;
    return RVE_OK;
  }
  ++S.restarts;
  // restart from the kept iterate (x = 0 if none was kept)
  if (S.have_best) CK(cudaMemcpyAsync(kv.x, xbest, vbytes, cudaMemcpyDeviceToDevice, h->stream));
  else CK(cudaMemsetAsync(kv.x, 0, vbytes, h->stream));
  KrylovScalars kk = k;
  kk.xE = S.have_best ? S.xE_best : 0.0;
  kk.done = 0;
  kk.status = 0;
  CK(cudaMemcpyAsync(h->ks, &kk, sizeof kk, cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  TRY((apply_scaled<TK, M>(h, kv.x, &h->ks->xE, kv.t, 0, 0, nullptr, nullptr, nullptr, nullptr, h->ks)));
  k_kresid<TK><<<h->Gpw, 256, 0, h->stream>>>(kv.len, bsave, kv.t, kv.r, h->part.kv);
  k_kfin_resid<<<1, 256, 0, h->stream>>>(h->ks, h->part.app, Gx, h->part.kv, h->Gpw);
  k_kinit<TK><<<h->Gpw, 256, 0, h->stream>>>(kv, S.restarts, 0);
  k_kfin_init<<<1, 256, 0, h->stream>>>(h->ks, h->part.kv, h->Gpw, kv.len, S.restarts, 0);
  h->launches += 4;
  CKL();
  return RVE_OK;
}

// end of a solve (on h->stream): the best iterate after a failed solve; outputs
template <typename TK, int M>
static int kry_end(rve *h, int *iters, int *status, double *relres) {
  KState &S = h->kst;
  if (S.st == 2) {
    TK *x = (TK *)h->kv[0], *xbest = (TK *)h->kv[8];
    const size_t vbytes = sizeof(TK) * (size_t)h->c * h->g.n;
    if (S.have_best) {
      CK(cudaMemcpyAsync(x, xbest, vbytes, cudaMemcpyDeviceToDevice, h->stream));
      h->ks_h->xE = S.xE_best;
    } else {
      CK(cudaMemsetAsync(x, 0, vbytes, h->stream));
      h->ks_h->xE = 0.0;
    }
    S.rel = S.bn > 0 ? S.rn_best / S.bn : 0.0;
  }
  *iters = S.total;
  *status = S.st;
  *relres = S.rel;
  return RVE_OK;
}

// The kernels of one chunk of BiCGStab iterations for nm RVEs of one shape and precision
// (a group of one for a single RVE): each pass is one launch over all members, the blocks
// of member i at blockIdx.y == i (the finalisers at blockIdx.x == i).
// Optional for float32 chunks (RVE_MERGED_UPDATE=1): BiCGStab's x / r update
// (x += alpha p + omega s, r = s - omega t) merged into the next iteration's x-forward pass,
// with |r|^2 and (rhat, r) taken from dots of s and t (krylov_fin.cuh fin_omega_conv): one
// pointwise pass less per iteration, 6 launches instead of 7, and only when every member's
// Krylov tolerance is at least 1e-4, far above the rounding of those expanded dots.  Off by
// default: on 512^2 composites the batched step ran at 66.7 increments/s with it against 70.9
// without (the x-forward pass, latency bound, pays more for the extra streams than the
// separate bandwidth-bound k_kxr pass costs).
template <typename TK>
static bool merged_update() {
  static const bool on = [] {
    const char *e = getenv("RVE_MERGED_UPDATE");
    return e && e[0] == '1';
  }();
  return sizeof(TK) == 4 && on;
}

template <typename TK, int M>
static int issue_chunk_n(rve *const *mem, int nm, cudaStream_t st) {
  rve *h = mem[0];
  const bool dbl = sizeof(TK) == 8;
  const int P = dbl ? h->Px_d : h->Px;
  const int Gx = dbl ? h->Gx_d : h->Gx;
  const size_t smx = dbl ? h->smx_d : h->smx_k;
  ApplyGroup<TK> A1, A2;
  KvGroup<TK> K;
  memset((void *)&A1, 0, sizeof A1);
  memset((void *)&A2, 0, sizeof A2);
  memset((void *)&K, 0, sizeof K);
  cpx<TK> *spec[kGroupMax];
  const KrylovScalars *ksc[kGroupMax];
  // float32 solves with a loose inner tolerance merge the x / r update into the next
  // iteration's x-forward pass (see merged_update)
  bool merged = merged_update<TK>();
  for (int i = 0; i < nm; ++i) merged = merged && mem[i]->desc.krylov_tol >= 1e-4;
  for (int i = 0; i < nm; ++i) {
    rve *m = mem[i];
    const KvArgs<TK> kv = kv_args<TK>(m);
    A1.m[i] = apply_args<TK, M>(m, kv.p, &m->ks->pE, kv.v, merged ? 5 : 1, 1, kv.r, kv.v, kv.rhat,
                                merged ? kv.s : nullptr, m->ks);
    A2.m[i] = apply_args<TK, M>(m, kv.s, &m->ks->sE, kv.t, 2, merged ? 6 : 2, kv.r, kv.v, kv.rhat, kv.s, m->ks);
    // the x-inverse passes (and k_kxr) finalise the scalars in their last block
    A1.m[i].fin = merged ? 5 : 1;
    A2.m[i].fin = merged ? 6 : 2;
    A1.m[i].xs = kv.x;
    A1.m[i].t = kv.t;
    A1.m[i].ksw = A2.m[i].ksw = m->ks;
    A1.m[i].arrive = A2.m[i].arrive = m->arrive;
    K.m[i] = kv;
    K.m[i].arrive = m->arrive + (merged ? 2 : 1);
    spec[i] = (cpx<TK> *)m->spec;
    ksc[i] = m->ks;
  }
  const FftPlan plx = plan_of<TK>(h, 0);
  const dim3 gx(Gx, nm), gpw(h->Gpw, nm);
  const int Wy = dbl ? h->Wy_d : h->Wy, Wz = dbl ? h->Wz_d : h->Wz;
  const size_t smy = dbl ? h->smy_d : h->smy_k, smz = dbl ? h->smz_d : h->smz_k;
  for (int j = 0; j < krylov_chunk_len(); ++j) {
    row_kernel<TK, M, true>(ct_len(h, 0), P, merged ? 5 : 1)<<<gx, 256, smx, st>>>(A1, plx, P);
    TRY((launch_columns_n<TK, M>(h, spec, ksc, nm, Wy, Wz, smy, smz, st)));
    row_kernel<TK, M, false>(ct_len(h, 0), P, 1)<<<gx, 256, smx, st>>>(A1, plx, P);  // + alpha
    row_kernel<TK, M, true>(ct_len(h, 0), P, 2)<<<gx, 256, smx, st>>>(A2, plx, P);
    TRY((launch_columns_n<TK, M>(h, spec, ksc, nm, Wy, Wz, smy, smz, st)));
    // + omega (merged: + convergence, the x / r update left pending)
    row_kernel<TK, M, false>(ct_len(h, 0), P, merged ? 6 : 2)<<<gx, 256, smx, st>>>(A2, plx, P);
    if (!merged) k_kxr<TK><<<gpw, 256, 0, st>>>(K);                          // + convergence
    h->launches += merged ? 4 : 5;
    CKL();
  }
  if (merged) {  // the last iteration's pending x / r update, so the host sees a whole iterate
    k_kx_finish<TK><<<gpw, 256, 0, st>>>(K);
    h->launches += 1;
    CKL();
  }
  return RVE_OK;
}

template <typename TK, int M>
static int krylov_group(rve *h, int *iters, int *status, double *relres);

template <typename TK, int M>
static int krylov_t(rve *h, int *iters, int *status, double *relres) {
  TRY((kry_begin<TK, M>(h)));
  if (h->kgroup) return krylov_group<TK, M>(h, iters, status, relres);
  // the chunk is a fixed kernel sequence over fixed buffers (every per-solve scalar lives in
  // device memory), captured once per handle and replayed: one graph launch per chunk
  if (!h->kgraph && graphs_enabled()) {
    if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    const long long l0 = h->launches;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    rve *one[1] = {h};
    int rc = e == cudaSuccess ? issue_chunk_n<TK, M>(one, 1, h->cap_stream) : RVE_E_CUDA;
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &graph);
    h->kgraph_launches = (int)(h->launches - l0);
    h->launches = l0;
    if (rc == RVE_OK && e2 == cudaSuccess && graph) {
      if (cudaGraphInstantiate(&h->kgraph, graph, 0) != cudaSuccess) h->kgraph = nullptr;
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
  }
  while (!h->kst.finished) {
    if (h->kgraph) {
      CK(cudaGraphLaunch(h->kgraph, h->stream));
      h->launches += h->kgraph_launches;
    } else {
      rve *one[1] = {h};
      TRY((issue_chunk_n<TK, M>(one, 1, h->stream)));
    }
    CK(cudaMemcpyAsync(h->ks_h, h->ks, sizeof(KrylovScalars), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    TRY((kry_after_chunk<TK, M>(h)));
  }
  return kry_end<TK, M>(h, iters, status, relres);
}

// ---- group execution of the Krylov solves of a batch ---------------------------------------
// RVEs of one shape, precision and tile schedule in rve_batch_crack_increment share a KGroup.
// Each runs its Newton loop on its own thread; at a Krylov solve it joins the group and
// waits.  One waiting member at a time leads: it runs chunks of BiCGStab iterations for every
// member in a solve (up to kGroupMax) as single launches per pass on the group stream,
// applies each member's after-chunk rule, admits newly waiting members at chunk boundaries
// and hands the lead over when its own solve is done.  A member's arithmetic is the same as
// alone (same kernels, blocks and reduction order), so its results are bit-identical.
struct KGroup {
  std::mutex mu;
  std::condition_variable cv;
  std::vector<rve *> pending, running;
  rve *leader = nullptr;
  cudaStream_t stream = nullptr;
};

// members per grouped launch (RVE_GROUP_MAX, 1..kGroupMax; default 4: with 16 RVEs of one
// shape, four groups keep four chunk streams in flight, as fast as one stream per RVE and
// with a quarter of the launches)
static int group_max() {
  static const int g = [] {
    const char *e = getenv("RVE_GROUP_MAX");
    const int v = e ? atoi(e) : 4;
    return v >= 1 && v <= kGroupMax ? v : kGroupMax;
  }();
  return g;
}

template <typename TK, int M>
static int group_lead(KGroup *G, std::unique_lock<std::mutex> &lk, rve *me) {
  for (;;) {
    while (!G->pending.empty() && (int)G->running.size() < group_max()) {
      G->running.push_back(G->pending.front());
      G->pending.erase(G->pending.begin());
    }
    if (G->running.empty()) {
      G->leader = nullptr;
      return RVE_OK;
    }
    std::vector<rve *> batch = G->running;
    lk.unlock();
    int rc = issue_chunk_n<TK, M>(batch.data(), (int)batch.size(), G->stream);
    for (rve *m : batch) {
      if (rc != RVE_OK) break;
      if (cudaMemcpyAsync(m->ks_h, m->ks, sizeof(KrylovScalars), cudaMemcpyDeviceToHost, G->stream) != cudaSuccess)
        rc = RVE_E_CUDA;
    }
    if (rc == RVE_OK && cudaStreamSynchronize(G->stream) != cudaSuccess) rc = RVE_E_CUDA;
    bool any_done = false;
    for (rve *m : batch) {
      // a waiting member's own stream is idle: its after-chunk work runs in order on the
      // group stream
      cudaStream_t own = m->stream;
      m->stream = G->stream;
      int r = rc == RVE_OK ? kry_after_chunk<TK, M>(m) : rc;
      m->stream = own;
      if (r != RVE_OK) {
        m->kst.finished = true;
        m->krc = r;
      }
      any_done = any_done || m->kst.finished;
    }
    if (any_done && cudaStreamSynchronize(G->stream) != cudaSuccess) rc = RVE_E_CUDA;
    lk.lock();
    for (size_t i = 0; i < G->running.size();) {
      rve *m = G->running[i];
      if (m->kst.finished || rc != RVE_OK) {
        if (rc != RVE_OK) m->krc = rc;
        m->kdone = true;
        G->running.erase(G->running.begin() + i);
      } else {
        ++i;
      }
    }
    G->cv.notify_all();
    if (me->kdone) {  // hand the lead to a member still waiting
      G->leader = nullptr;
      G->cv.notify_all();
      return RVE_OK;
    }
  }
}

template <typename TK, int M>
static int krylov_group(rve *h, int *iters, int *status, double *relres) {
  KGroup *G = h->kgroup;
  CK(cudaStreamSynchronize(h->stream));  // kry_begin's work is done before the group uses it
  {
    std::unique_lock<std::mutex> lk(G->mu);
    h->kdone = false;
    h->krc = RVE_OK;
    G->pending.push_back(h);
    while (!h->kdone) {
      if (G->leader == nullptr) {
        G->leader = h;
        group_lead<TK, M>(G, lk, h);
        continue;
      }
      G->cv.wait_for(lk, std::chrono::milliseconds(1));
    }
  }
  if (h->krc != RVE_OK) return h->krc;
  return kry_end<TK, M>(h, iters, status, relres);
}

static int krylov(rve *h, int *iters, int *status, double *relres) {
  if (h->mixed) {
    if (h->m == 3) return krylov_t<float, 3>(h, iters, status, relres);
    return krylov_t<float, 6>(h, iters, status, relres);
  }
  if (h->m == 3) return krylov_t<double, 3>(h, iters, status, relres);
  return krylov_t<double, 6>(h, iters, status, relres);
}

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// RVE_VERBOSE=1 in the environment traces every Newton iteration on stderr.
static bool verbose() {
  static int v = -1;
  if (v < 0) {
    const char *e = getenv("RVE_VERBOSE");
    v = (e && e[0] && e[0] != '0') ? 1 : 0;
  }
  return v == 1;
}

static double rel_or(double a, double b) {
  if (a == 0.0) return 0.0;
  return b > 0.0 ? a / b : INFINITY;
}

// eps_tilde <- G : eps_tilde (float64 FFT round trip, in place)
template <int M>
static int project_strain_t(rve *h, double *eps) {
  ResidArgs ra;
  memset(&ra, 0, sizeof ra);
  ra.g = h->g;
  ra.sigma = eps;
  ra.phi = eps;  // the extra channel is transformed and discarded
  ra.spec = (cpx<double> *)h->spec;
  k_xfwd_resid<M><<<h->Gx_d, 256, h->smx_d, h->stream>>>(ra, plan_of<double>(h, 0), h->Px_d);
  h->launches += 1;
  CKL();
  TRY((launch_columns<double, M>(h, ra.spec, nullptr, h->Wy_d, h->Wz_d, h->smy_d, h->smz_d)));
  k_xinv_proj<M><<<h->Gx_d, 256, h->smx_d, h->stream>>>(ra, plan_of<double>(h, 0), h->Px_d, eps);
  h->launches += 1;
  CKL();
  return RVE_OK;
}

static int project_strain(rve *h, double *eps) {
  return h->m == 3 ? project_strain_t<3>(h, eps) : project_strain_t<6>(h, eps);
}

// Newton step update of the working state; returns the step error terms
// Float32 runs: the strain part of a Newton step goes through the Galerkin projection in
// float32 (kv[7] = G : x_eps) before it is added, so the float64 eps_tilde stays compatible
// up to float32 rounding of the step itself; float64 runs project eps_tilde after the update.
template <int M>
static int project_step_f32_t(rve *h) {
  ApplyArgs<float> a;
  memset(&a, 0, sizeof a);
  a.g = h->g;
  a.x = (float *)h->kv[0];
  a.y = (float *)h->kv[7];
  a.tan = (const float *)h->tan;
  a.xE_ptr = h->red + 40;
  a.e_scale = 0.0;
  a.spec = (cpx<float> *)h->spec;
  a.part = h->part.app;
  a.pro_mode = 4;
  a.epi_mode = 3;
  a.tr = spec_tr<float, M>(h);
  row_kernel<float, M, true>(ct_len(h, 0), h->Px, a.pro_mode)<<<h->Gx, 256, h->smx_k, h->stream>>>(solo(a), plan_of<float>(h, 0), h->Px);
  h->launches += 1;
  CKL();
  TRY((launch_columns<float, M>(h, a.spec, nullptr, h->Wy, h->Wz, h->smy_k, h->smz_k)));
  row_kernel<float, M, false>(ct_len(h, 0), h->Px, a.epi_mode)<<<h->Gx, 256, h->smx_k, h->stream>>>(solo(a), plan_of<float>(h, 0), h->Px);
  h->launches += 1;
  CKL();
  return RVE_OK;
}
static int project_step_f32(rve *h) {
  return h->m == 3 ? project_step_f32_t<3>(h) : project_step_f32_t<6>(h);
}

static int newton_update(rve *h, double step, double xE, double *err_step) {
  const double E_new = h->E_w + step * xE;
  const size_t mn = (size_t)h->m * h->g.n;
  if (h->mixed)
    k_newton_update<float><<<h->Gpw, 256, 0, h->stream>>>(h->g.n, h->m, (const float *)h->kv[7],
                                                           (const float *)h->kv[0] + mn, step,
                                                           h->eps_w, h->phi_w, h->fM_d, E_new, h->part.upd);
  else
    k_newton_update<double><<<h->Gpw, 256, 0, h->stream>>>(h->g.n, h->m, (const double *)h->kv[0],
                                                            (const double *)h->kv[0] + mn, step,
                                                            h->eps_w, h->phi_w, h->fM_d, E_new, h->part.upd);
  h->launches += 1;
  CKL();
  double u[4];
  TRY(reduce_to_host(h, h->part.upd, h->Gpw, 4, 0, u));
  const double dE = step * xE;
  h->E_w = E_new;
  const double e_eps = rel_or(fabs(step) * sqrt(u[0]), sqrt(u[2]));
  const double e_E = rel_or(fabs(dE), fabs(h->E_w));
  const double e_phi = rel_or(fabs(step) * sqrt(u[1]), sqrt(u[3]));
  if (!(isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]) && isfinite(u[3]) && isfinite(h->E_w)))
    return RVE_E_NOCONV;
  *err_step = fmax(e_eps, fmax(e_E, e_phi));
  h->last_e_eps = e_eps;
  h->last_e_phi = e_phi;
  return RVE_OK;
}

// |S J e_E|: apply to x = 0, x_E = 1 (device scratch vectors), norm of the result
template <typename TK, int M>
static int column_norm_E_t(rve *h, double *out) {
  const long long len = (long long)h->c * h->g.n;
  TK *x = (TK *)h->kv[5], *t = (TK *)h->kv[6];
  CK(cudaMemsetAsync(x, 0, sizeof(TK) * len, h->stream));
  const double one = 1.0;
  CK(cudaMemcpyAsync(h->red + 40, &one, sizeof(double), cudaMemcpyHostToDevice, h->stream));
  const double keep = h->e_scale;
  h->e_scale = 1.0;
  TRY((apply_scaled<TK, M>(h, x, h->red + 40, t, 0, 0, nullptr, nullptr, nullptr, nullptr, nullptr)));
  h->e_scale = keep;
  k_norm2<TK><<<h->Gpw, 256, 0, h->stream>>>(len, t, h->part.kv);
  h->launches += 1;
  CKL();
  const int Gx = sizeof(TK) == 8 ? h->Gx_d : h->Gx;
  double aw[2];
  ReduceList L;
  memset(&L, 0, sizeof L);
  L.s[0] = {h->part.kv, h->Gpw, 1, 0, 0};
  L.s[1] = {h->part.app, Gx, 1, 0, 0};
  L.n = 2;
  TRY(reduce_list_to_host(h, L, aw));
  const double yE = h->lin_s3 * aw[1];
  *out = sqrt(aw[0] + yE * yE);
  return RVE_OK;
}

static int column_norm_E(rve *h, double *out) {
  if (h->mixed) {
    if (h->m == 3) return column_norm_E_t<float, 3>(h, out);
    return column_norm_E_t<float, 6>(h, out);
  }
  if (h->m == 3) return column_norm_E_t<double, 3>(h, out);
  return column_norm_E_t<double, 6>(h, out);
}

// ---- tile-schedule autotuner -------------------------------------------------------------
// Times the Krylov-precision operator apply for candidate (P row pairs per x-pass block,
// W columns per column-pass block) and keeps the fastest.  Values of the operands do not
// matter for the timing; scratch vectors are zeroed first.
template <typename TK, int M>
static int autotune_t(rve *h) {
  const long long len = (long long)h->c * h->g.n;
  TK *x = (TK *)h->kv[5], *y = (TK *)h->kv[6];
  CK(cudaMemsetAsync(x, 0, sizeof(TK) * len, h->stream));
  CK(cudaMemsetAsync(h->red + 40, 0, sizeof(double), h->stream));
  const int es = sizeof(TK);
  const int Ps[4] = {1, 2, 4, 8}, Ws[5] = {1, 2, 4, 8, 16};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int bP = h->Px, bW = h->Wy;
  // The candidates are timed as solo applies, but the batched step runs the float32 2D passes
  // of several RVEs concurrently as grouped launches.  On 512^2 composites the step ran at
  // 59.3-59.8 increments/s with P = 1, 63.5-64.1 with P = 2 and 57.7 with P = 4, while the
  // solo apply ranks them differently from box to box (within 3-5 %); P = 4 also leaves a
  // grouped launch of four RVEs at half a wave.  Likewise the fused column pass: with 4, 2 and
  // 1 columns per block (W = 1, 2, 4) a grouped apply of four took 69.4, 67.9 and 64.6 us and
  // the step ran at 68.5, 71.6 and 73.4 increments/s, yet the solo timing picked 4 columns on
  // some boxes.  Float32 2D grids of at least 256 x 256 therefore take P = 2 and W = 4
  // untimed; narrower rows (where larger P fills a block) are tuned.
  const bool fix_p2 = sizeof(TK) == 4 && h->g.d == 2 && h->g.rows >= 256 && h->g.nx >= 256;
  for (int pi = 0; pi < 4; ++pi)
    for (int wi = 0; wi < 5; ++wi) {
      int P, Gx, Wy, Wz;
      size_t smx, smy, smz;
      if (fix_p2 && (Ps[pi] != 2 || Ws[wi] != 4)) continue;
      pass_geometry(h->g, es, Ps[pi], Ws[wi], P, Gx, Wy, Wz, smx, smy, smz);
      // clamped: covered by another candidate (the fixed schedule takes its clamped form)
      if (!fix_p2 && (P != Ps[pi] || Wy != Ws[wi])) continue;
      h->Px = P; h->Gx = Gx; h->Wy = Wy; h->Wz = Wz; h->smx_k = smx; h->smy_k = smy; h->smz_k = smz;
      if (sizeof(TK) == 8) {
        h->Px_d = P; h->Gx_d = Gx; h->Wy_d = Wy; h->Wz_d = Wz; h->smx_d = smx; h->smy_d = smy; h->smz_d = smz;
      }
      TRY((apply_scaled<TK, M>(h, x, h->red + 40, y, 0, 0, nullptr, nullptr, nullptr, nullptr, nullptr)));
      CK(cudaEventRecord(e0, h->stream));
      for (int r = 0; r < 3; ++r)
        TRY((apply_scaled<TK, M>(h, x, h->red + 40, y, 0, 0, nullptr, nullptr, nullptr, nullptr, nullptr)));
      CK(cudaEventRecord(e1, h->stream));
      CK(cudaEventSynchronize(e1));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        bP = P;
        bW = Wy;
      }
    }
  pass_geometry(h->g, es, bP, bW, h->Px, h->Gx, h->Wy, h->Wz, h->smx_k, h->smy_k, h->smz_k);
  if (sizeof(TK) == 8)
    pass_geometry(h->g, 8, bP, bW, h->Px_d, h->Gx_d, h->Wy_d, h->Wz_d, h->smx_d, h->smy_d, h->smz_d);
  // Radix plan per axis, with the chosen tiles: each distinct variant of a length that has
  // no compile-time kernel (the compile-time kernels run variant 0 with every index folded,
  // which a runtime-length kernel does not beat) is timed as a solo apply, and the fastest
  // kept.  The column axis of the fused 2D pass keeps variant 0.  Float32 (MIXED) handles
  // only: a choice made by timing changes the rounding from machine to machine, which the
  // float64 solver, the reference for the stored oracle runs, should not do.
  if (forced_plan_variant() < 0 && sizeof(TK) == 4) {
    for (int a = 0; a < h->g.d; ++a) {
      const int N = a == 0 ? h->g.nx : (a == 1 ? h->g.ny : h->g.nz);
      if (has_ct_kernel(N, h->m) || (a == 1 && h->tr)) continue;
      const std::vector<int> vs = distinct_variants(N);
      if (vs.size() < 2) continue;
      float bt = 1e30f;
      int bv = h->pvar[a];
      for (int v : vs) {
        TRY(set_plan_variant(h, a, v));
        TRY((apply_scaled<TK, M>(h, x, h->red + 40, y, 0, 0, nullptr, nullptr, nullptr, nullptr, nullptr)));
        CK(cudaEventRecord(e0, h->stream));
        for (int r = 0; r < 3; ++r)
          TRY((apply_scaled<TK, M>(h, x, h->red + 40, y, 0, 0, nullptr, nullptr, nullptr, nullptr, nullptr)));
        CK(cudaEventRecord(e1, h->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < bt) {
          bt = ms;
          bv = v;
        }
      }
      TRY(set_plan_variant(h, a, bv));
      if (verbose()) fprintf(stderr, "[rve] autotune: axis %d length %d plan variant %d apply %.1f us\n", a, N, bv, 1e3 * bt / 3);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->tuned = 1;
  if (h->kgraph) {
    cudaGraphExecDestroy(h->kgraph);
    h->kgraph = nullptr;
  }
  if (verbose()) fprintf(stderr, "[rve] autotune: P %d W %d apply %.1f us\n", bP, bW, 1e3 * best / 3);
  return RVE_OK;
}

// Tiles and plan variants chosen per (grid, precision) in this process: later handles of the
// same shape reuse them, so equal problems run with equal reduction orders (bit-identical
// results).
#include <map>
#include <mutex>
#include <tuple>
struct TuneRecord {
  int P, W, pvar[3];
};
static std::map<std::tuple<int, int, int, int>, TuneRecord> g_tiles;
static std::mutex g_tiles_mu;

static void apply_tiles(rve *h, int P, int W) {
  if (h->kgraph) {
    cudaGraphExecDestroy(h->kgraph);
    h->kgraph = nullptr;
  }
  const int es = h->mixed ? 4 : 8;
  pass_geometry(h->g, es, P, W, h->Px, h->Gx, h->Wy, h->Wz, h->smx_k, h->smy_k, h->smz_k);
  if (!h->mixed) pass_geometry(h->g, 8, P, W, h->Px_d, h->Gx_d, h->Wy_d, h->Wz_d, h->smx_d, h->smy_d, h->smz_d);
  h->tuned = 1;
}

static int apply_record(rve *h, const TuneRecord &r) {
  apply_tiles(h, r.P, r.W);
  for (int a = 0; a < 3; ++a)
    if (h->pvar[a] != r.pvar[a]) TRY(set_plan_variant(h, a, r.pvar[a]));
  return RVE_OK;
}

static int autotune(rve *h) {
  const auto key = std::make_tuple(h->g.nx, h->g.ny, h->g.nz, h->mixed);
  {
    // RVE_TILES="P,W" fixes the tile schedule (row pairs per x-pass block, kx columns per
    // column-pass block) instead of timing candidates
    const char *e = getenv("RVE_TILES");
    int P = 0, W = 0;
    if (e && sscanf(e, "%d,%d", &P, &W) == 2 && P > 0 && W > 0) {
      apply_tiles(h, P, W);
      return RVE_OK;
    }
  }
  if (forced_plan_variant() >= 0) {  // plans fixed by the environment: tiles timed, nothing shared
    if (h->mixed) return h->m == 3 ? autotune_t<float, 3>(h) : autotune_t<float, 6>(h);
    return h->m == 3 ? autotune_t<double, 3>(h) : autotune_t<double, 6>(h);
  }
  {
    TuneRecord rec;
    bool found = false;
    {
      std::lock_guard<std::mutex> lk(g_tiles_mu);
      auto it = g_tiles.find(key);
      if (it != g_tiles.end()) {
        rec = it->second;
        found = true;
      }
    }
    if (found) return apply_record(h, rec);
  }
  if (h->mixed) TRY(h->m == 3 ? (autotune_t<float, 3>(h)) : (autotune_t<float, 6>(h)));
  else TRY(h->m == 3 ? (autotune_t<double, 3>(h)) : (autotune_t<double, 6>(h)));
  TuneRecord mine{h->Px, h->Wy, {h->pvar[0], h->pvar[1], h->pvar[2]}}, rec;
  {
    std::lock_guard<std::mutex> lk(g_tiles_mu);
    auto it = g_tiles.find(key);
    if (it == g_tiles.end()) {
      g_tiles[key] = mine;
      return RVE_OK;
    }
    rec = it->second;  // another thread won
  }
  return apply_record(h, rec);
}

static bool autotune_enabled() {
  const char *e = getenv("RVE_AUTOTUNE");
  return !(e && e[0] == '0');
}

struct NewtonOut {
  int converged, iters, kry, applies;
  double err;
  double sum_eps, sum_phi;  // relative eps / phi change summed over the Newton steps
};

// Algorithm 2 inner loop on the working state (eps_w, phi_w, E_w) with history H^n = Hn.
static int newton(rve *h, int control, double target, NewtonOut *no) {
  memset(no, 0, sizeof *no);
  const double floor_ = 1e-13;
  double prev_step_err = INFINITY;
  int prev_exact = 0;
  // err of the step before the last one when that was an exact step (else infinite): the
  // observed contraction theta = err / err_hist < 0.5 accepts an iterate whose estimated
  // error theta / (1 - theta) * err is within the tolerance (same rule as the oracle)
  double err_hist = INFINITY;
  // backtracking (same rule as the oracle): a step that grew the scaled residual norm more
  // than 1.5-fold is halved in place, up to 6 times
  const double kLsGrowth = 1.5;
  const int kLsMax = 6;
  double bn_prev = 0.0, last_step = 0.0, last_xE = 0.0;
  bool have_last = false;
  int halvings = 0;
  if (!h->tuned && autotune_enabled()) TRY(autotune(h));
  for (int it = 1;; ++it) {
    double t0 = now_s();
    TRY(linearize(h, h->eps_w, h->phi_w, h->E_w, control, target));
    h->t_phase[0] += now_s() - t0;
    if (have_last && isfinite(h->lin_bn2) && sqrt(h->lin_bn2) > kLsGrowth * bn_prev && halvings < kLsMax) {
      const double hs = 0.5 * last_step;
      int rc = newton_update(h, -hs, last_xE, &prev_step_err);
      if (rc != RVE_OK) return rc;
      if (!h->mixed) TRY(project_strain(h, h->eps_w));
      last_step = hs;
      ++halvings;
      prev_step_err = INFINITY;  // a backtracked step never ends the loop
      err_hist = INFINITY;
      if (verbose()) fprintf(stderr, "[rve]   backtrack: step %.3e\n", hs);
      --it;
      continue;
    }
    if (have_last && !isfinite(h->lin_bn2) && halvings < kLsMax) {
      const double hs = 0.5 * last_step;
      int rc = newton_update(h, -hs, last_xE, &prev_step_err);
      if (rc != RVE_OK) return rc;
      if (!h->mixed) TRY(project_strain(h, h->eps_w));
      last_step = hs;
      ++halvings;
      prev_step_err = INFINITY;
      err_hist = INFINITY;
      --it;
      continue;
    }
    halvings = 0;
    if (verbose())
      fprintf(stderr, "[rve] newton %d ctrl %d E %.15e Gamma %.15e target %.15e |b| %.3e ref %.3e step_err %.3e exact %d\n",
              it, control, h->E_w, h->lin_gamma, target, sqrt(h->lin_bn2), h->lin_ref, prev_step_err, prev_exact);
    if (!isfinite(h->lin_bn2) || !isfinite(h->lin_cval)) {
      set_err(h, "non-finite residual");
      return RVE_E_NOCONV;
    }
    if (it > 1) {
      double err = prev_step_err;
      if (control == RVE_CTRL_CRACK) err = fmax(err, rel_or(fabs(h->lin_cval - target), fabs(target)));
      no->err = err;
      double est = err;
      if (prev_exact && isfinite(err_hist) && err_hist > 0.0) {
        const double th = err / err_hist;
        if (th < 0.5) est = fmin(err, th / (1.0 - th) * err);
      }
      if (sqrt(h->lin_bn2) <= floor_ * h->lin_ref || (prev_exact && est <= h->desc.newton_tol)) {
        no->converged = 1;
        no->iters = it - 1;
        return RVE_OK;
      }
      err_hist = prev_exact ? err : INFINITY;
    }
    if (it > h->desc.newton_max) {
      set_err(h, "Newton did not converge in %d iterations (err %.3e)", h->desc.newton_max, no->err);
      return RVE_E_NOCONV;
    }
    // column scaling of the E unknown (crack control): |S J e_E| = 0.1
    h->e_scale = 1.0;
    t0 = now_s();
    if (control == RVE_CTRL_CRACK) {
      double cn = 0;
      TRY(column_norm_E(h, &cn));
      no->applies += 1;
      if (cn > 0) h->e_scale = 0.1 / cn;
    }
    CK(cudaMemcpyAsync(&h->ks->escale, &h->e_scale, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    h->t_phase[1] += now_s() - t0;
    int kits = 0, kst = 0;
    double krel = 0;
    t0 = now_s();
    TRY(krylov(h, &kits, &kst, &krel));
    h->t_phase[2] += now_s() - t0;
    t0 = now_s();
    no->kry += kits;
    no->applies += 2 * kits;
    prev_exact = kst == 0;
    if (verbose())
      fprintf(stderr, "[rve]   krylov its %d status %d rel %.3e e_scale %.3e xE %.6e\n", kits, kst, krel,
              h->e_scale, h->ks_h->xE);
    if (kst != 0 && !(krel < 0.5)) {
      set_err(h, "BiCGStab failed (status %d, relative residual %.3e after %d iterations)", kst, krel, kits);
      return RVE_E_NOCONV;
    }
    // step length: alpha, bounded under crack control so that E at most doubles or halves,
    // and so that no phase-field value moves by more than 1 (same rule as the oracle)
    const double xE = h->ks_h->xE * h->e_scale;
    double step = h->desc.alpha;
    if (control == RVE_CTRL_CRACK && xE != 0.0) {
      const double rho = xE > 0.0 ? 1.0 : 0.5;
      if (fabs(step * xE) > rho * fabs(h->E_w)) step = rho * fabs(h->E_w) / fabs(xE);
    }
    {
      const long long n = h->g.n;
      if (h->mixed) k_maxabs<float><<<h->Gpw, 256, 0, h->stream>>>(n, (const float *)h->kv[0] + h->m * n, h->part.cmax);
      else k_maxabs<double><<<h->Gpw, 256, 0, h->stream>>>(n, (const double *)h->kv[0] + h->m * n, h->part.cmax);
      h->launches += 1;
      CKL();
      double dpmax = 0;
      TRY(reduce_to_host(h, h->part.cmax, h->Gpw, 1, 1, &dpmax));
      if (dpmax > 0.0 && step * dpmax > 1.0) step = 1.0 / dpmax;
    }
    bn_prev = sqrt(h->lin_bn2);
    if (h->mixed) TRY(project_step_f32(h));
    int rc = newton_update(h, step, xE, &prev_step_err);
    if (rc != RVE_OK) {
      set_err(h, "non-finite Newton update");
      return rc;
    }
    if (!h->mixed) TRY(project_strain(h, h->eps_w));
    h->t_phase[3] += now_s() - t0;
    no->sum_eps += h->last_e_eps;
    no->sum_phi += h->last_e_phi;
    have_last = true;
    last_step = step;
    last_xE = xE;
  }
}

// ---- state management ----------------------------------------------------------------------
static int copy_committed_to_work(rve *h) {
  const size_t n = h->g.n;
  CK(cudaMemcpyAsync(h->eps_w, h->eps_c, sizeof(double) * h->m * n, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(h->phi_w, h->phi_c, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
  h->E_w = h->E_c;
  return RVE_OK;
}
static int commit_work(rve *h, double tau) {
  const size_t n = h->g.n;
  std::swap(h->eps_w, h->eps_c);
  std::swap(h->phi_w, h->phi_c);
  // history: H^{n+1} = max(psi+, H^n) evaluated at the converged state (Eq. history)
  CK(cudaMemcpyAsync(h->Hn, h->Hcur, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
  h->E_c = h->E_w;
  h->tau_c = tau;
  return RVE_OK;
}

static void fill_step(rve *h, const NewtonOut &no, rve_step *out) {
  if (!out) return;
  memset(out, 0, sizeof *out);
  out->E = h->E_c;
  for (int k = 0; k < h->m; ++k) out->sigma[k] = h->lin_sigma_sum[k] / (double)h->g.n;
  out->gamma = h->lin_gamma;
  out->tau = h->tau_c;
  out->newton_iters = no.iters;
  out->krylov_iters = no.kry;
  out->applies = no.applies;
  out->err = no.err;
}

static int strain_solve(rve *h, double E_target, NewtonOut *no) {
  TRY(copy_committed_to_work(h));
  int rc = newton(h, RVE_CTRL_STRAIN, E_target, no);
  return rc;
}

// ================================ C ABI ======================================================
extern "C" {

void rve_desc_defaults(rve_desc *d) {
  memset(d, 0, sizeof *d);
  d->nz = 1;
  d->ell = 2.0;
  d->f[1] = 1.0;
  d->split = RVE_SPLIT_SPECTRAL;
  d->precision = RVE_FP64;
  d->k_res = 0.0;
  d->alpha = 1.0;
  d->newton_tol = 1e-10;
  d->krylov_tol = 1e-10;
  d->newton_max = 50;
  d->krylov_max = 4000;
}

const char *rve_last_error(const rve_t *h) { return h ? h->err.c_str() : g_err; }

// Pinned host mirrors (reduction outputs, Krylov scalars) come from a process-wide free list
// and go back to it: cudaFreeHost would synchronise the device.
static std::mutex g_pinned_mu;
static std::vector<void *> g_pinned_free;  // blocks of kPinnedBytes
static constexpr size_t kPinnedBytes = 8 * 64 > sizeof(KrylovScalars) ? 8 * 64 : sizeof(KrylovScalars);

static void *pinned_get() {
  {
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    if (!g_pinned_free.empty()) {
      void *p = g_pinned_free.back();
      g_pinned_free.pop_back();
      return p;
    }
  }
  void *p = nullptr;
  if (cudaMallocHost(&p, kPinnedBytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

static void pinned_put(void *p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pinned_mu);
  g_pinned_free.push_back(p);
}

static void free_all(rve *h) {
  if (!h) return;
  // stream-ordered frees after the handle's last work; a handle without a stream of its own
  // frees on the legacy stream and waits for it (memory is back in the pool on return)
  cudaStream_t fs = h->stream;
#define cudaFree(ptr) cudaFreeAsync((ptr), fs)
  void *ptrs[] = {h->mat, h->eps_c, h->phi_c, h->Hn, h->eps_w, h->phi_w, h->sigma, h->Hcur, h->F,
                  h->Lphi, h->s2, h->fM_d, h->spec, h->tan, h->ks, h->arrive, h->red, h->ext_dq, h->en,
                  h->part.cons, h->tw_d[0], h->tw_d[1], h->tw_d[2], h->tw_f[0], h->tw_f[1], h->tw_f[2]};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (int i = 0; i < 9; ++i)
    if (h->kv[i]) cudaFree(h->kv[i]);
  for (int a = 0; a < 3; ++a)
    if (h->perm[a]) cudaFree(h->perm[a]);
  for (int a = 0; a < 3; ++a)
    for (int t = 0; t < 3; ++t) {
      if (h->tabs_d[a][t]) cudaFree(h->tabs_d[a][t]);
      if (h->tabs_f[a][t]) cudaFree(h->tabs_f[a][t]);
    }
#undef cudaFree
  if (!fs) cudaStreamSynchronize(0);
  pinned_put(h->red_h);
  pinned_put(h->ks_h);
  h->red_h = nullptr;
  h->ks_h = nullptr;
}

void rve_destroy(rve_t *h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  {
    const char *e = getenv("RVE_TIMING");  // "1": host seconds per Newton phase on stderr
    if (e && e[0] == '1')
      fprintf(stderr, "[rve] timing: linearize %.3f s, E column %.3f s, krylov %.3f s, update %.3f s\n",
              h->t_phase[0], h->t_phase[1], h->t_phase[2], h->t_phase[3]);
  }
  if (h->kgraph) cudaGraphExecDestroy(h->kgraph);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->twin) {
    h->twin->stream = nullptr;  // shares the handle's stream
    rve_destroy(h->twin);
    h->twin = nullptr;
  }
  free_all(h);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

static int dalloc(rve *h, void **p, size_t bytes) {
  if (h->fault_alloc_at > 0 && ++h->alloc_calls == h->fault_alloc_at) {
    *p = nullptr;
    set_err(h, "device allocation of %zu bytes failed: injected by RVE_FAULT", bytes);
    return RVE_E_OOM;
  }
  // stream-ordered allocation from the device's memory pool (on the legacy stream, which
  // rve_create's synchronous copies follow): freeing it later (cudaFreeAsync on the handle's
  // stream) does not synchronise the whole device, so a server that retires an RVE does not
  // stall the other resident RVEs' streams
  cudaError_t e = cudaMallocAsync(p, bytes, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_err(h, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    return RVE_E_OOM;
  }
  return RVE_OK;
}

static int create_impl(const rve_desc *d, rve *h) {
  if (!d || d->nx < 1 || d->ny < 1 || d->nz < 1 || d->n_phases < 1 || d->n_phases > RVE_MAX_PHASES ||
      !d->phase || !d->E || !d->nu || !d->Gc || !(d->ell > 0) ||
      (d->precision != RVE_FP64 && d->precision != RVE_MIXED) ||
      (d->split != RVE_SPLIT_SPECTRAL && d->split != RVE_SPLIT_NONE) ||
      (d->gamma_op != RVE_GAMMA_ROTATED && d->gamma_op != RVE_GAMMA_CONTINUOUS) ||
      (d->constraint != RVE_CONSTRAINT_LENGTH && d->constraint != RVE_CONSTRAINT_ENERGY) || d->newton_max < 1 ||
      d->krylov_max < 1 || !(d->alpha > 0)) {
    set_err(h, "invalid rve_desc (sizes, phases, ell > 0, precision, split, limits)");
    return RVE_E_ARG;
  }
  {
    const char *fe = getenv("RVE_FAULT");
    h->fault_alloc_at = (fe && strncmp(fe, "alloc:", 6) == 0) ? atoi(fe + 6) : 0;
    h->fault_breakdown = (fe && strcmp(fe, "krylov_breakdown") == 0) ? 1 : 0;
    h->alloc_calls = 0;
  }
  h->desc = *d;
  h->desc.phase = nullptr;
  h->desc.E = h->desc.nu = h->desc.Gc = nullptr;
  Geo &g = h->g;
  g.nx = d->nx;
  g.ny = d->ny;
  g.nz = d->nz;
  g.d = d->nz == 1 ? 2 : 3;
  g.m = g.d == 2 ? 3 : 6;
  g.c = g.m + 1;
  g.hx = g.nx / 2 + 1;
  g.rows = g.ny * g.nz;
  g.n = (long long)g.nx * g.ny * g.nz;
  h->dim = g.d;
  h->m = g.m;
  h->c = g.c;
  h->mixed = d->precision == RVE_MIXED;
  {
    const char *e = getenv("RVE_FUSED_COLUMNS");  // "0" keeps the unfused column pass
    const bool want = !(e && e[0] == '0');
    bool ct = false;
    for (int li = 0; li < 5; ++li) ct = ct || g.ny == kCtLengths[li];
    h->tr = (want && h->mixed && g.nz == 1 && ct) ? 1 : 0;
  }
  h->n_phases = d->n_phases;
  const long long n = g.n;
  h->phase_host.assign(d->phase, d->phase + n);
  h->E_ph.assign(d->E, d->E + d->n_phases);
  h->nu_ph.assign(d->nu, d->nu + d->n_phases);
  h->Gc_ph.assign(d->Gc, d->Gc + d->n_phases);
  memset(&h->ph, 0, sizeof h->ph);
  h->C_ref = 0;
  for (int p = 0; p < d->n_phases; ++p) {
    const double E = d->E[p], nu = d->nu[p];
    if (!(E > 0) || !(nu > -1.0 && nu < 0.5) || !(d->Gc[p] > 0)) {
      set_err(h, "phase %d: need E > 0, -1 < nu < 0.5, Gc > 0", p);
      return RVE_E_ARG;
    }
    h->ph.lam[p] = E * nu / ((1 + nu) * (1 - 2 * nu));
    h->ph.mu[p] = E / (2 * (1 + nu));
    h->ph.Gc[p] = d->Gc[p];
    h->C_ref = fmax(h->C_ref, h->ph.lam[p] + 2 * h->ph.mu[p]);
  }
  for (long long v = 0; v < n; ++v)
    if (d->phase[v] >= d->n_phases) {
      set_err(h, "phase id %d at voxel %lld out of range", (int)d->phase[v], v);
      return RVE_E_ARG;
    }
  h->s1 = 1.0 / h->C_ref;
  for (int k = 0; k < 6; ++k) h->fM[k] = k < g.m ? d->f[k] : 0.0;
  // mean |xi|^2 over the grid = sum over axes of the per-axis mean of xi_a^2
  h->Lbar = 0;
  const int ext[3] = {g.nx, g.ny, g.nz};
  for (int a = 0; a < g.d; ++a) {
    const int N = ext[a];
    double s = 0;
    for (int k = 0; k < N; ++k) {
      const int ks = (2 * k < N) ? k : k - N;
      const double xi = 2.0 * M_PI * ks / N;
      s += xi * xi;
    }
    h->Lbar += s / N;
  }
  h->stream = 0;
  TRY(make_plan(h, g.nx, h->plx, &h->tw_d[0], &h->tw_f[0], &h->perm[0]));
  TRY(make_plan(h, g.ny, h->ply, &h->tw_d[1], &h->tw_f[1], &h->perm[1]));
  TRY(make_plan(h, g.nz, h->plz, &h->tw_d[2], &h->tw_f[2], &h->perm[2]));
  for (int a = 0; a < 3; ++a) TRY(make_axis_tables(h, a, ext[a], d->gamma_op));
  {
    const int fv = forced_plan_variant();
    if (fv > 0)
      for (int a = 0; a < g.d; ++a) {
        if (a == 1 && h->tr) continue;
        const std::vector<int> vs = distinct_variants(ext[a]);
        if (std::find(vs.begin(), vs.end(), fv) != vs.end()) TRY(set_plan_variant(h, a, fv));
      }
  }
  // launch geometry
  const int esk = h->mixed ? 4 : 8;
  pass_geometry(g, esk, 0, 0, h->Px, h->Gx, h->Wy, h->Wz, h->smx_k, h->smy_k, h->smz_k);
  pass_geometry(g, 8, 0, 0, h->Px_d, h->Gx_d, h->Wy_d, h->Wz_d, h->smx_d, h->smy_d, h->smz_d);
  if ((long long)(g.m == 3 ? TanIdx<3>::K : TanIdx<6>::K) * g.n >= (1LL << 31)) {
    set_err(h, "grid of %lld voxels exceeds the 32-bit channel indexing of the kernels", g.n);
    return RVE_E_ARG;
  }
  {
    size_t need = h->smx_k;
    const size_t cand[5] = {h->smy_k, h->smz_k, h->smx_d, h->smy_d, h->smz_d};
    for (size_t v : cand) need = v > need ? v : need;
    TRY(set_smem_attrs(h, need));
  }
  // pointwise Krylov kernels (grid-stride loops): about 16 vector elements per thread, at
  // least two and at most eight blocks of 256 threads per SM, never more blocks than voxels /
  // 256.  The upper bound keeps the float32 per-thread dot sums short (with two blocks per SM
  // the 128^3 porous solve needed 20 % more BiCGStab iterations and its increments took 10 %
  // longer); the lower bound gives a 512^2 RVE 304 blocks rather than 1024 (single-RVE
  // increments 2.5 % faster: fewer partials for the last block to sum).  RVE_PW_BLOCKS
  // overrides the result.
  const long long gp = (n + 255) / 256;
  long long gw = ((long long)g.c * n + 4095) / 4096;
  gw = gw < 152 * 2 ? 152 * 2 : (gw > 152 * 8 ? 152 * 8 : gw);
  {
    const char *e = getenv("RVE_PW_BLOCKS");  // 1 .. 1216 (the footprint's bound)
    if (e && atoi(e) > 0) gw = atoi(e) < 152 * 8 ? atoi(e) : 152 * 8;
  }
  h->Gpw = (int)(gp < gw ? gp : gw);
  // memory
  const size_t m = g.m, c = g.c;
  const size_t tk = h->mixed ? 4 : 8;
  const int K = g.m == 3 ? TanIdx<3>::K : TanIdx<6>::K;
  TRY(dalloc(h, (void **)&h->mat, n));
  TRY(dalloc(h, (void **)&h->eps_c, 8 * m * n));
  TRY(dalloc(h, (void **)&h->eps_w, 8 * m * n));
  TRY(dalloc(h, (void **)&h->phi_c, 8 * n));
  TRY(dalloc(h, (void **)&h->phi_w, 8 * n));
  TRY(dalloc(h, (void **)&h->Hn, 8 * n));
  TRY(dalloc(h, (void **)&h->sigma, 8 * m * n));
  TRY(dalloc(h, (void **)&h->Hcur, 8 * n));
  TRY(dalloc(h, (void **)&h->F, 8 * c * n));
  TRY(dalloc(h, (void **)&h->Lphi, 8 * n));
  TRY(dalloc(h, (void **)&h->s2, 8 * n));
  TRY(dalloc(h, (void **)&h->fM_d, 8 * 6));
  TRY(dalloc(h, (void **)&h->spec, 16 * c * (size_t)g.rows * g.hx));
  TRY(dalloc(h, (void **)&h->tan, tk * K * n));
  for (int i = 0; i < 9; ++i) TRY(dalloc(h, &h->kv[i], tk * c * n));
  TRY(dalloc(h, (void **)&h->ks, sizeof(KrylovScalars)));
  TRY(dalloc(h, (void **)&h->arrive, 4 * sizeof(unsigned int)));
  CK(cudaMemset(h->arrive, 0, 4 * sizeof(unsigned int)));
  TRY(dalloc(h, (void **)&h->red, 8 * 64));
  TRY(dalloc(h, (void **)&h->ext_dq, 8 * (c * n + 1)));
  // partial buffers sized for the smallest x-pass tile (one row pair per block)
  const int Gx_max = (g.rows + 1) / 2;
  const int Gm = h->Gpw > Gx_max ? h->Gpw : Gx_max;
  double *pb = nullptr;
  TRY(dalloc(h, (void **)&pb, 8 * (size_t)Gm * 28));
  h->part.cons = pb;
  h->part.cmax = pb + 8 * (size_t)Gm;
  h->part.res = pb + 9 * (size_t)Gm;
  h->part.app = pb + 14 * (size_t)Gm;
  h->part.kv = pb + 20 * (size_t)Gm;
  h->part.upd = pb + 22 * (size_t)Gm;
  h->part.en = pb + 26 * (size_t)Gm;
  if (d->constraint == RVE_CONSTRAINT_ENERGY) {
    TRY(dalloc(h, (void **)&h->en, 8 * m * n));
    CK(cudaMemset(h->en, 0, 8 * m * n));
  }
  h->red_h = (double *)pinned_get();
  h->ks_h = (KrylovScalars *)pinned_get();
  if (!h->red_h || !h->ks_h) {
    set_err(h, "pinned host allocation failed");
    return RVE_E_OOM;
  }
  // initial state: eps_tilde = 0, E = 0, phi = 0, H = 0 (Algorithm 2 initial data)
  std::vector<uint8_t> matv(n);
  for (long long v = 0; v < n; ++v) matv[v] = d->phase[v];
  CK(cudaMemcpy(h->mat, matv.data(), n, cudaMemcpyHostToDevice));
  CK(cudaMemset(h->eps_c, 0, 8 * m * n));
  CK(cudaMemset(h->phi_c, 0, 8 * n));
  CK(cudaMemset(h->Hn, 0, 8 * n));
  CK(cudaMemcpy(h->fM_d, h->fM, 8 * 6, cudaMemcpyHostToDevice));
  CK(cudaMemset(h->tan, 0, tk * K * n));
  CK(cudaStreamSynchronize(0));  // the stream-ordered allocations are complete for any stream
  h->E_c = h->E_w = 0;
  h->tau_c = 0;
  h->started = 0;
  h->notch_set = 0;
  return RVE_OK;
}

// Device bytes rve_create allocates for a descriptor (solver buffers, spectral scratch,
// Krylov vectors, reduction partials, plans and tables).
static long long footprint_bytes(const rve_desc *d) {
  const long long nx = d->nx, ny = d->ny, nz = d->nz;
  const long long n = nx * ny * nz, rows = ny * nz, hx = nx / 2 + 1;
  const long long m = nz == 1 ? 3 : 6, c = m + 1;
  const long long tk = d->precision == RVE_MIXED ? 4 : 8;
  const long long K = nz == 1 ? TanIdx<3>::K : TanIdx<6>::K;
  long long gpw = (n + 255) / 256;  // upper bound of the handle's pointwise grid
  if (gpw > 152 * 8) gpw = 152 * 8;
  const long long gm = gpw > (rows + 1) / 2 ? gpw : (rows + 1) / 2;
  long long b = n;                          // material bytes
  b += 8 * (2 * m + 3 + m + 3 + c) * n;     // states, sigma, H, L phi, s2, F
  b += 16 * c * rows * hx;                  // spectral scratch
  b += tk * K * n + 9 * tk * c * n;         // tangent channels, Krylov vectors
  b += 8 * (c * n + 1) + 8 * 28 * gm;       // host-apply scratch, partials
  b += 16;                                  // arrival counters
  if (d->constraint == RVE_CONSTRAINT_ENERGY) b += 8 * m * n;  // energy-control work space
  b += (long long)(nx + ny + nz) * (16 + 8 + 4 + 3 * 12) + 4096;  // plans, tables, scalars
  return b;
}

// Eq. JaviGc: (area / length) * int Sigma:f dE over the load path by the trapezoid rule,
// starting from the unloaded state (0, 0).
int rve_effective_toughness(const double *E, const double *sigma_f, int n, double area, double length,
                            double *G) {
  if (!E || !sigma_f || !G || n < 0 || !(length > 0)) return RVE_E_ARG;
  double work = 0.0, e0 = 0.0, s0 = 0.0;
  for (int i = 0; i < n; ++i) {
    work += 0.5 * (sigma_f[i] + s0) * (E[i] - e0);
    e0 = E[i];
    s0 = sigma_f[i];
  }
  *G = area * work / length;
  return RVE_OK;
}

// J-integral of the committed state around the rectangle of voxel centres (x0, y0)-(x1, y1),
// 2D: rotation field from the strain fluctuation (float64 FFT passes and k_rot_spec), then the
// contour sum (k_j_contour).  Uses the spectral scratch and the stress buffer as work space.
int rve_j_integral(rve_t *h, int x0, int y0, int x1, int y1, double *J) {
  if (!h || !J) return RVE_E_ARG;
  const Geo &g = h->g;
  if (g.d != 2) {
    set_err(h, "rve_j_integral is defined for 2D grids only");
    return RVE_E_ARG;
  }
  if (x0 < 0 || y0 < 0 || x1 >= g.nx || y1 >= g.ny || x0 >= x1 || y0 >= y1) {
    set_err(h, "contour (%d, %d)-(%d, %d) is not a rectangle inside the %d x %d grid", x0, y0, x1, y1, g.nx,
            g.ny);
    return RVE_E_ARG;
  }
  ResidArgs ra;
  memset(&ra, 0, sizeof ra);
  ra.g = g;
  ra.sigma = h->eps_c;
  ra.phi = h->eps_c;  // the extra channel is transformed and discarded
  ra.spec = (cpx<double> *)h->spec;
  k_xfwd_resid<3><<<h->Gx_d, 256, h->smx_d, h->stream>>>(ra, plan_of<double>(h, 0), h->Px_d);
  CKL();
  ColGroup<double> G;
  memset((void *)&G, 0, sizeof G);
  ColArgs<double> &ca = G.base;
  ca.g = g;
  ca.spec = ra.spec;
  ca.tab = tabs_of<double>(h);
  ca.inv_n = 1.0 / (double)g.n;
  ca.yplan = plan_of<double>(h, 1);
  ca.axis = 1;
  ca.W = h->Wy_d;
  ca.lw = 0;
  while ((1 << ca.lw) < ca.W) ++ca.lw;
  ca.plan = plan_of<double>(h, 1);
  G.spec[0] = ra.spec;
  const dim3 grid((g.hx + h->Wy_d - 1) / h->Wy_d, 1, 1);
  col_kernel<double, 3, 0>(ct_len(h, 1))<<<grid, 256, h->smy_d, h->stream>>>(G);
  CKL();
  RotArgs rk;
  rk.g = g;
  rk.spec = ra.spec;
  rk.yrev = ca.plan.rev;
  rk.inv_n = 1.0 / (double)g.n;
  k_rot_spec<<<h->Gpw, 256, 0, h->stream>>>(rk);
  CKL();
  col_kernel<double, 3, 2>(ct_len(h, 1))<<<grid, 256, h->smy_d, h->stream>>>(G);
  CKL();
  k_xinv_proj<3><<<h->Gx_d, 256, h->smx_d, h->stream>>>(ra, plan_of<double>(h, 0), h->Px_d, h->sigma);
  CKL();
  h->lin_valid = 0;  // the stress buffer now holds the rotation field (channel 0)
  JArgs ja;
  memset(&ja, 0, sizeof ja);
  ja.g = g;
  ja.eps_t = h->eps_c;
  ja.phi = h->phi_c;
  ja.w = h->sigma;
  ja.mat = h->mat;
  ja.ph = h->ph;
  for (int k = 0; k < 3; ++k) ja.fM[k] = h->fM[k];
  ja.E = h->E_c;
  ja.k_res = h->desc.k_res;
  ja.isotropic = h->desc.split == RVE_SPLIT_NONE;
  ja.x0 = x0;
  ja.y0 = y0;
  ja.x1 = x1;
  ja.y1 = y1;
  ja.out = h->red + 48;
  k_j_contour<<<1, 256, 0, h->stream>>>(ja);
  CKL();
  CK(cudaMemcpyAsync(h->red_h + 48, h->red + 48, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *J = h->red_h[48];
  return RVE_OK;
}

int rve_footprint(const rve_desc *desc, long long *bytes) {
  if (!desc || !bytes || desc->nx < 1 || desc->ny < 1 || desc->nz < 1) return RVE_E_ARG;
  *bytes = footprint_bytes(desc);
  return RVE_OK;
}

int rve_create(const rve_desc *desc, rve_t **out) {
  if (!out) {
    set_err(nullptr, "out is NULL");
    return RVE_E_ARG;
  }
  *out = nullptr;
  rve *h = new rve();
  memset((void *)&h->g, 0, sizeof h->g);
  h->mat = nullptr;
  h->eps_c = h->phi_c = h->Hn = h->eps_w = h->phi_w = h->sigma = h->Hcur = h->F = h->Lphi = h->s2 = h->fM_d = nullptr;
  h->spec = nullptr;
  h->tan = nullptr;
  for (int i = 0; i < 9; ++i) h->kv[i] = nullptr;
  h->ks = nullptr;
  h->red = nullptr;
  h->red_h = nullptr;
  h->ks_h = nullptr;
  h->ext_dq = nullptr;
  h->en = nullptr;
  memset(&h->part, 0, sizeof h->part);
  memset(h->tabs_d, 0, sizeof h->tabs_d);
  memset(h->tabs_f, 0, sizeof h->tabs_f);
  memset(h->t_phase, 0, sizeof h->t_phase);
  memset(h->tw_d, 0, sizeof h->tw_d);
  memset(h->tw_f, 0, sizeof h->tw_f);
  memset(h->perm, 0, sizeof h->perm);
  h->launches = 0;
  h->lin_valid = 0;
  h->e_scale = 1.0;
  h->tuned = 0;
  h->own_stream = 0;
  h->cap_stream = nullptr;
  h->kgraph = nullptr;
  h->kgraph_launches = 0;
  h->kgroup = nullptr;
  h->twin = nullptr;
  h->fp64_left = 0;
  h->fault_alloc_at = h->alloc_calls = h->fault_breakdown = 0;
  h->stag_mode = 0;
  h->last_e_eps = h->last_e_phi = 0.0;
  h->kdone = false;
  h->krc = 0;
  int rc = create_impl(desc, h);
  if (rc != RVE_OK) {
    snprintf(g_err, sizeof g_err, "%s", h->err.c_str());
    rve_destroy(h);
    return rc;
  }
  *out = h;
  return RVE_OK;
}

int rve_autotune(rve_t *h) {
  if (!h) return RVE_E_ARG;
  TRY(autotune(h));
  CK(cudaStreamSynchronize(h->stream));
  return RVE_OK;
}

int rve_set_stream(rve_t *h, void *stream) {
  if (!h) return RVE_E_ARG;
  if (h->own_stream && h->stream) {
    cudaStreamSynchronize(h->stream);
    cudaStreamDestroy(h->stream);
  }
  h->own_stream = 0;
  h->stream = (cudaStream_t)stream;
  return RVE_OK;
}

int rve_info(const rve_t *h, int *dim, int *m, long long *n, int *precision) {
  if (!h) return RVE_E_ARG;
  if (dim) *dim = h->dim;
  if (m) *m = h->m;
  if (n) *n = h->g.n;
  if (precision) *precision = h->desc.precision;
  return RVE_OK;
}

long long rve_kernel_launches(const rve_t *h) { return h ? h->launches : 0; }

int rve_set_notch(rve_t *h, const uint8_t *mask) {
  if (!h || !mask) return RVE_E_ARG;
  if (h->started) {
    set_err(h, "rve_set_notch after the first increment");
    return RVE_E_STATE;
  }
  const long long n = h->g.n;
  std::vector<uint8_t> matv(n);
  std::vector<double> phi(n);
  for (long long v = 0; v < n; ++v) {
    matv[v] = h->phase_host[v] | (mask[v] ? RVE_NOTCH_BIT : 0);
    phi[v] = mask[v] ? 1.0 : 0.0;
  }
  CK(cudaMemcpy(h->mat, matv.data(), n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->phi_c, phi.data(), 8 * n, cudaMemcpyHostToDevice));
  h->notch_set = 1;
  return RVE_OK;
}

int rve_startup(rve_t *h, double beta, rve_step *out) {
  if (!h) return RVE_E_ARG;
  if (h->started) {
    set_err(h, "already started");
    return RVE_E_STATE;
  }
  if (!(beta > 0)) beta = 0.25;
  NewtonOut no;
  int tot_k = 0, tot_n = 0, tot_a = 0;
  // (a) E = 0: phase-field profile of the notch
  TRY(strain_solve(h, 0.0, &no));
  TRY(commit_work(h, 0.0));
  tot_k += no.kry;
  tot_n += no.iters;
  tot_a += no.applies;
  // (b) probe load
  double gmin = INFINITY;
  for (int p = 0; p < h->n_phases; ++p) gmin = fmin(gmin, h->ph.Gc[p] / h->desc.ell);
  const double Ep = 1e-3 * sqrt(gmin / h->C_ref);
  TRY(strain_solve(h, Ep, &no));
  tot_k += no.kry;
  tot_n += no.iters;
  tot_a += no.applies;
  const double ratio = h->lin_maxratio;  // evaluated at the converged probe state
  if (!(ratio > 0)) {
    set_err(h, "load direction produces no tensile energy");
    return RVE_E_ARG;
  }
  // keep the probe state as the start of (c) but with history still H = 0
  std::swap(h->eps_w, h->eps_c);
  std::swap(h->phi_w, h->phi_c);
  h->E_c = h->E_w;
  const double Es = Ep * sqrt(beta / ratio);
  TRY(strain_solve(h, Es, &no));
  tot_k += no.kry;
  tot_n += no.iters;
  tot_a += no.applies;
  TRY(commit_work(h, h->lin_cval));
  // (d) strain-controlled loading E <- 1.25 E, history committed each step, until Gamma has
  // grown by 0.5 over its value at (c) or a step fails to converge (same rule as the oracle)
  const double g0 = h->lin_gamma;
  double gam = g0, cval = h->lin_cval;
  for (int k = 0; k < 40 && gam - g0 < 0.5; ++k) {
    int rc = strain_solve(h, h->E_c * 1.25, &no);
    if (rc == RVE_E_NOCONV) break;  // the committed state is untouched
    if (rc != RVE_OK) return rc;
    tot_k += no.kry;
    tot_n += no.iters;
    tot_a += no.applies;
    TRY(commit_work(h, h->lin_cval));
    gam = h->lin_gamma;
    cval = h->lin_cval;
  }
  h->tau_c = cval;
  h->started = 1;
  no.kry = tot_k;
  no.iters = tot_n;
  no.applies = tot_a;
  fill_step(h, no, out);
  return RVE_OK;
}

// One increment with cut-back (same rule as the oracle): a failed Newton solve is retried
// as two committed half increments, recursively down to da / 8.
static int crack_increment_cb(rve *h, double da, int depth, NewtonOut *acc, int *cutbacks) {
  TRY(copy_committed_to_work(h));
  const double tau = h->tau_c + da;
  NewtonOut no;
  int rc = newton(h, RVE_CTRL_CRACK, tau, &no);
  acc->iters += no.iters;
  acc->kry += no.kry;
  acc->applies += no.applies;
  acc->err = no.err;
  if (rc == RVE_OK) return commit_work(h, tau);
  if (rc != RVE_E_NOCONV || depth >= 3) return rc;
  if (verbose()) fprintf(stderr, "[rve] cut-back: da %.4g -> 2 x %.4g\n", da, 0.5 * da);
  *cutbacks += 1;
  // keep the committed state to restore it if the halves fail too
  const size_t n = h->g.n, m = h->m;
  std::vector<double> eps(m * n), phi(n), H(n);
  CK(cudaMemcpyAsync(eps.data(), h->eps_c, 8 * m * n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(phi.data(), h->phi_c, 8 * n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(H.data(), h->Hn, 8 * n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const double E0 = h->E_c, tau0 = h->tau_c;
  rc = crack_increment_cb(h, 0.5 * da, depth + 1, acc, cutbacks);
  if (rc == RVE_OK) rc = crack_increment_cb(h, 0.5 * da, depth + 1, acc, cutbacks);
  if (rc != RVE_OK) {
    CK(cudaMemcpyAsync(h->eps_c, eps.data(), 8 * m * n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->phi_c, phi.data(), 8 * n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->Hn, H.data(), 8 * n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->E_c = E0;
    h->tau_c = tau0;
  }
  return rc;
}

// increments that stay on the float64 twin after a fallback (RVE_FP64_STICKY, default 0)
static int fp64_sticky() {
  static const int k = [] {
    const char *e = getenv("RVE_FP64_STICKY");
    return e ? atoi(e) : 0;
  }();
  return k;
}

static bool fp64_fallback_enabled() {
  static const bool on = [] {
    const char *e = getenv("RVE_FP64_FALLBACK");  // "0": a failed mixed increment stays failed
    return !(e && e[0] == '0');
  }();
  return on;
}

// The committed state of a handle (eps_tilde, phi, H^n, E, tau) copied to another handle of the
// same grid, on the destination's stream after the source's work.
static int copy_committed(rve *dst, const rve *src) {
  rve *h = dst;
  const size_t n = src->g.n, m = src->m;
  CK(cudaStreamSynchronize(src->stream));
  CK(cudaMemcpyAsync(dst->eps_c, src->eps_c, 8 * m * n, cudaMemcpyDeviceToDevice, dst->stream));
  CK(cudaMemcpyAsync(dst->phi_c, src->phi_c, 8 * n, cudaMemcpyDeviceToDevice, dst->stream));
  CK(cudaMemcpyAsync(dst->Hn, src->Hn, 8 * n, cudaMemcpyDeviceToDevice, dst->stream));
  CK(cudaStreamSynchronize(dst->stream));
  dst->E_c = src->E_c;
  dst->tau_c = src->tau_c;
  dst->started = 1;
  dst->lin_valid = 0;
  return RVE_OK;
}

// Redo a crack increment of a RVE_MIXED handle in float64 (iterative refinement of the whole
// increment: the float32 inner solves could not contract the float64 Newton residual, which
// happens where the bordered system is badly conditioned).  The twin is a float64 handle of
// the same RVE, created on first use and kept; it starts from the handle's committed state
// and, on success, its committed state becomes the handle's.
static int fp64_twin_increment(rve *h, double da, rve_step *st) {
  if (!h->twin) {
    rve_desc d = h->desc;
    d.precision = RVE_FP64;
    d.krylov_tol = 1e-10;
    d.phase = h->phase_host.data();
    d.E = h->E_ph.data();
    d.nu = h->nu_ph.data();
    d.Gc = h->Gc_ph.data();
    rve_t *t = nullptr;
    const int rc = rve_create(&d, &t);
    if (rc != RVE_OK) {
      set_err(h, "float64 fallback: %s", rve_last_error(nullptr));
      return rc;
    }
    t->stream = h->stream;
    CK(cudaMemcpyAsync(t->mat, h->mat, (size_t)h->g.n, cudaMemcpyDeviceToDevice, h->stream));
    t->notch_set = h->notch_set;
    h->twin = t;
  }
  rve *t = h->twin;
  t->stream = h->stream;
  TRY(copy_committed(t, h));
  const int rc = rve_crack_increment(t, da, st);
  if (rc != RVE_OK) {
    set_err(h, "float64 fallback: %s", t->err.c_str());
    return rc;
  }
  TRY(copy_committed(h, t));
  return RVE_OK;
}

int rve_crack_increment(rve_t *h, double da, rve_step *out) {
  if (!h) return RVE_E_ARG;
  if (!h->started) TRY(rve_startup(h, 0.25, nullptr));
  NewtonOut acc;
  memset(&acc, 0, sizeof acc);
  int cutbacks = 0;
  int rc = RVE_E_NOCONV;
  if (h->fp64_left > 0) --h->fp64_left;  // this increment goes to the twin directly
  else rc = crack_increment_cb(h, da, 0, &acc, &cutbacks);
  if (rc == RVE_E_NOCONV && h->mixed && fp64_fallback_enabled()) {
    if (h->fp64_left == 0 && acc.iters > 0) h->fp64_left = fp64_sticky();
    if (verbose()) fprintf(stderr, "[rve] mixed increment failed: float64 fallback\n");
    rve_step st;
    memset(&st, 0, sizeof st);
    rc = fp64_twin_increment(h, da, &st);
    if (rc != RVE_OK) return rc;
    h->last_applies = 4 * (st.applies + acc.applies);  // float64 applies cost about 4 float32 ones
    if (out) {
      *out = st;
      out->newton_iters += acc.iters;
      out->krylov_iters += acc.kry;
      out->applies += acc.applies;
      out->cutbacks += cutbacks;
      out->fallbacks = 1;
    }
    return RVE_OK;
  }
  if (rc != RVE_OK) return rc;
  h->last_applies = acc.applies;
  fill_step(h, acc, out);
  if (out) out->cutbacks = cutbacks;
  return RVE_OK;
}

int rve_strain_increment(rve_t *h, double E_target, rve_step *out) {
  if (!h) return RVE_E_ARG;
  NewtonOut no;
  TRY(strain_solve(h, E_target, &no));
  TRY(commit_work(h, h->lin_cval));
  h->started = 1;
  fill_step(h, no, out);
  return RVE_OK;
}

int rve_staggered_increment(rve_t *h, double E_target, double tol, int max_sweeps, rve_step *out,
                            int *sweeps) {
  if (!h || !(tol > 0) || max_sweeps < 1) return RVE_E_ARG;
  TRY(copy_committed_to_work(h));
  NewtonOut tot;
  memset(&tot, 0, sizeof tot);
  int sw = 0, rc = RVE_OK;
  bool conv = false;
  for (sw = 1; sw <= max_sweeps; ++sw) {
    NewtonOut n1, n2;
    h->stag_mode = 1;  // mechanics at fixed phi
    rc = newton(h, RVE_CTRL_STRAIN, E_target, &n1);
    if (rc != RVE_OK) break;
    h->stag_mode = 2;  // phase field at fixed H = max(psi+, H^n)
    rc = newton(h, RVE_CTRL_STRAIN, E_target, &n2);
    if (rc != RVE_OK) break;
    tot.iters += n1.iters + n2.iters;
    tot.kry += n1.kry + n2.kry;
    tot.applies += n1.applies + n2.applies;
    tot.err = fmax(n1.sum_eps, n2.sum_phi);
    if (tot.err <= tol) {
      conv = true;
      break;
    }
  }
  h->stag_mode = 0;
  if (rc != RVE_OK) return rc;  // the committed state is unchanged
  if (!conv) {
    set_err(h, "staggered iteration did not converge in %d sweeps (change %.3e)", max_sweeps, tot.err);
    return RVE_E_NOCONV;
  }
  TRY(commit_work(h, h->lin_cval));
  h->started = 1;
  tot.converged = 1;
  fill_step(h, tot, out);
  if (sweeps) *sweeps = sw;
  return RVE_OK;
}

int rve_get_macro_stress(const rve_t *hc, double sigma[6], double *E) {
  rve *h = (rve *)hc;
  if (!h) return RVE_E_ARG;
  // evaluate sigma at the committed state
  TRY(linearize(h, h->eps_c, h->phi_c, h->E_c, RVE_CTRL_STRAIN, h->E_c));
  h->lin_valid = 0;
  if (sigma)
    for (int k = 0; k < 6; ++k) sigma[k] = k < h->m ? h->lin_sigma_sum[k] / (double)h->g.n : 0.0;
  if (E) *E = h->E_c;
  return RVE_OK;
}

int rve_get_fields(const rve_t *hc, int which, double *dst, size_t count) {
  rve *h = (rve *)hc;
  if (!h || !dst) return RVE_E_ARG;
  const size_t n = h->g.n, m = h->m;
  switch (which) {
    case RVE_FIELD_EPS: {
      if (count < m * n) return RVE_E_ARG;
      k_total_strain<<<h->Gpw, 256, 0, h->stream>>>(n, h->m, h->eps_c, h->fM_d, h->E_c, h->sigma);
      CKL();
      CK(cudaMemcpyAsync(dst, h->sigma, 8 * m * n, cudaMemcpyDeviceToHost, h->stream));
      break;
    }
    case RVE_FIELD_EPS_T:
      if (count < m * n) return RVE_E_ARG;
      CK(cudaMemcpyAsync(dst, h->eps_c, 8 * m * n, cudaMemcpyDeviceToHost, h->stream));
      break;
    case RVE_FIELD_PHI:
      if (count < n) return RVE_E_ARG;
      CK(cudaMemcpyAsync(dst, h->phi_c, 8 * n, cudaMemcpyDeviceToHost, h->stream));
      break;
    case RVE_FIELD_H:
      if (count < n) return RVE_E_ARG;
      CK(cudaMemcpyAsync(dst, h->Hn, 8 * n, cudaMemcpyDeviceToHost, h->stream));
      break;
    case RVE_FIELD_SIGMA:
      if (count < m * n) return RVE_E_ARG;
      TRY(linearize(h, h->eps_c, h->phi_c, h->E_c, RVE_CTRL_STRAIN, h->E_c));
      h->lin_valid = 0;
      CK(cudaMemcpyAsync(dst, h->sigma, 8 * m * n, cudaMemcpyDeviceToHost, h->stream));
      break;
    default:
      set_err(h, "unknown field %d", which);
      return RVE_E_ARG;
  }
  CK(cudaStreamSynchronize(h->stream));
  return RVE_OK;
}

int rve_set_state(rve_t *h, const double *eps_tilde, const double *phi, const double *H, double E,
                  double tau) {
  if (!h || !eps_tilde || !phi || !H) return RVE_E_ARG;
  const size_t n = h->g.n, m = h->m;
  // a non-finite value would poison every later solve: reject it before any device copy
  if (!isfinite(E) || !isfinite(tau)) {
    set_err(h, "rve_set_state: E or tau is not finite");
    return RVE_E_ARG;
  }
  const double *arrs[3] = {eps_tilde, phi, H};
  const size_t lens[3] = {m * n, n, n};
  for (int a = 0; a < 3; ++a) {
    // x * 0 is NaN exactly when x is not finite; eight independent sums keep the loop from
    // waiting on a single chain of additions (the states of a 512^2 RVE are 1.3 M values)
    double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const double *x = arrs[a];
    size_t i = 0;
    for (; i + 8 <= lens[a]; i += 8)
      for (int k = 0; k < 8; ++k) acc[k] += x[i + k] * 0.0;
    for (; i < lens[a]; ++i) acc[0] += x[i] * 0.0;
    double tot = 0.0;
    for (int k = 0; k < 8; ++k) tot += acc[k];
    if (tot != 0.0) {
      set_err(h, "rve_set_state: %s holds a non-finite value", a == 0 ? "eps_tilde" : (a == 1 ? "phi" : "H"));
      return RVE_E_ARG;
    }
  }
  CK(cudaMemcpy(h->eps_c, eps_tilde, 8 * m * n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->phi_c, phi, 8 * n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->Hn, H, 8 * n, cudaMemcpyHostToDevice));
  h->E_c = E;
  h->tau_c = tau;
  h->started = 1;
  h->lin_valid = 0;
  return RVE_OK;
}

int rve_linearize(rve_t *h, int control, double target) {
  if (!h || (control != RVE_CTRL_CRACK && control != RVE_CTRL_STRAIN)) return RVE_E_ARG;
  TRY(copy_committed_to_work(h));
  TRY(linearize(h, h->eps_w, h->phi_w, h->E_w, control, target));
  CK(cudaStreamSynchronize(h->stream));
  return RVE_OK;
}

int rve_residual(const rve_t *hc, double *F1, double *F2, double *F3) {
  rve *h = (rve *)hc;
  if (!h) return RVE_E_ARG;
  if (!h->lin_valid) {
    set_err(h, "rve_residual needs rve_linearize first");
    return RVE_E_STATE;
  }
  const size_t n = h->g.n, m = h->m;
  if (F1) CK(cudaMemcpyAsync(F1, h->F, 8 * m * n, cudaMemcpyDeviceToHost, h->stream));
  if (F2) CK(cudaMemcpyAsync(F2, h->F + m * n, 8 * n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (F3) *F3 = h->lin_F3;
  return RVE_OK;
}

int rve_apply_device(rve_t *h, const void *x, const double *xE, void *y, double *yE) {
  if (!h || !x || !xE || !y || !yE) return RVE_E_ARG;
  if (!h->lin_valid) {
    set_err(h, "rve_apply_device needs rve_linearize first");
    return RVE_E_STATE;
  }
  h->launches = 0;
  if (h->mixed) {
    if (h->m == 3) TRY((apply_scaled<float, 3>(h, (float *)x, xE, (float *)y, 0, 0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, yE)));
    else TRY((apply_scaled<float, 6>(h, (float *)x, xE, (float *)y, 0, 0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, yE)));
  } else {
    if (h->m == 3) TRY((apply_scaled<double, 3>(h, (double *)x, xE, (double *)y, 0, 0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, yE)));
    else TRY((apply_scaled<double, 6>(h, (double *)x, xE, (double *)y, 0, 0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, yE)));
  }
  return RVE_OK;
}

}  // extern "C"

template <typename TK, int M>
static int apply_batch_t(rve *const *hs, int n, const void *const *x, const double *const *xE, void *const *y,
                         double *const *yE) {
  rve *h = hs[0];
  cudaStream_t st = h->stream;
  const bool dbl = sizeof(TK) == 8;
  const int P = dbl ? h->Px_d : h->Px;
  const int Gx = dbl ? h->Gx_d : h->Gx;
  const size_t smx = dbl ? h->smx_d : h->smx_k;
  ApplyGroup<TK> A;
  memset((void *)&A, 0, sizeof A);
  cpx<TK> *spec[kGroupMax];
  const KrylovScalars *ks[kGroupMax];
  for (int i = 0; i < n; ++i) {
    A.m[i] = apply_args<TK, M>(hs[i], (TK *)x[i], xE[i], (TK *)y[i], 0, 0, nullptr, nullptr, nullptr, nullptr,
                               nullptr);
    A.m[i].fin = hs[i]->lin_control == RVE_CTRL_STRAIN ? 4 : 3;  // E slot of y in the x-inverse pass
    A.m[i].yE = yE[i];
    spec[i] = (cpx<TK> *)hs[i]->spec;
    ks[i] = nullptr;
  }
  const dim3 gx(Gx, n);
  row_kernel<TK, M, true>(ct_len(h, 0), P, A.m[0].pro_mode)<<<gx, 256, smx, st>>>(A, plan_of<TK>(h, 0), P);
  h->launches += 1;
  CKL();
  TRY((launch_columns_n<TK, M>(h, spec, ks, n, dbl ? h->Wy_d : h->Wy, dbl ? h->Wz_d : h->Wz,
                               dbl ? h->smy_d : h->smy_k, dbl ? h->smz_d : h->smz_k, st)));
  row_kernel<TK, M, false>(ct_len(h, 0), P, A.m[0].epi_mode)<<<gx, 256, smx, st>>>(A, plan_of<TK>(h, 0), P);
  h->launches += 1;
  CKL();
  return RVE_OK;
}

extern "C" {

int rve_apply_device_batch(rve_t *const *hs, int count, const void *const *x, const double *const *xE,
                           void *const *y, double *const *yE) {
  if (!hs || !x || !xE || !y || !yE || count < 1 || count > kGroupMax || !hs[0]) return RVE_E_ARG;
  rve *h = hs[0];
  for (int i = 0; i < count; ++i) {
    rve *o = hs[i];
    if (!o || !x[i] || !xE[i] || !y[i] || !yE[i]) return RVE_E_ARG;
    if (o->g.nx != h->g.nx || o->g.ny != h->g.ny || o->g.nz != h->g.nz || o->mixed != h->mixed ||
        o->Px != h->Px || o->Wy != h->Wy || o->Wz != h->Wz || o->Px_d != h->Px_d || o->Wy_d != h->Wy_d ||
        o->Wz_d != h->Wz_d || o->tr != h->tr || o->pvar[0] != h->pvar[0] || o->pvar[1] != h->pvar[1] ||
        o->pvar[2] != h->pvar[2]) {
      set_err(h, "rve_apply_device_batch: RVE %d differs from RVE 0 in shape, precision, tiles or FFT plans", i);
      return RVE_E_ARG;
    }
    if (!o->lin_valid) {
      set_err(h, "rve_apply_device_batch: RVE %d needs rve_linearize first", i);
      return RVE_E_STATE;
    }
  }
  h->launches = 0;
  if (h->mixed) {
    if (h->m == 3) return apply_batch_t<float, 3>(hs, count, x, xE, y, yE);
    return apply_batch_t<float, 6>(hs, count, x, xE, y, yE);
  }
  if (h->m == 3) return apply_batch_t<double, 3>(hs, count, x, xE, y, yE);
  return apply_batch_t<double, 6>(hs, count, x, xE, y, yE);
}

int rve_apply(rve_t *h, const double *dq_eps, const double *dq_phi, double dq_E, double *out_eps,
              double *out_phi, double *out_E) {
  if (!h || !dq_eps || !dq_phi || !out_eps || !out_phi || !out_E) return RVE_E_ARG;
  if (!h->lin_valid) {
    set_err(h, "rve_apply needs rve_linearize first");
    return RVE_E_STATE;
  }
  const size_t n = h->g.n, m = h->m, c = h->c;
  double *d = h->ext_dq;
  CK(cudaMemcpyAsync(d, dq_eps, 8 * m * n, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(d + m * n, dq_phi, 8 * n, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(d + c * n, &dq_E, 8, cudaMemcpyHostToDevice, h->stream));
  // x -> Krylov slot 0 in the Krylov precision, y in slot 4; the E slot of y in red[32]
  if (h->mixed) k_convert<double, float><<<h->Gpw, 256, 0, h->stream>>>(c * n, d, (float *)h->kv[0]);
  else k_convert<double, double><<<h->Gpw, 256, 0, h->stream>>>(c * n, d, (double *)h->kv[0]);
  CKL();
  TRY(rve_apply_device(h, h->kv[0], d + c * n, h->kv[4], h->red + 32));
  std::vector<double> y(c * n), s2(n);
  if (h->mixed) {
    k_convert<float, double><<<h->Gpw, 256, 0, h->stream>>>(c * n, (const float *)h->kv[4], d);
    CKL();
    CK(cudaMemcpyAsync(y.data(), d, 8 * c * n, cudaMemcpyDeviceToHost, h->stream));
  } else {
    CK(cudaMemcpyAsync(y.data(), h->kv[4], 8 * c * n, cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaMemcpyAsync(s2.data(), h->s2, 8 * n, cudaMemcpyDeviceToHost, h->stream));
  double yE = 0;
  CK(cudaMemcpyAsync(&yE, h->red + 32, 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (size_t i = 0; i < m * n; ++i) out_eps[i] = y[i] / h->s1;
  for (size_t v = 0; v < n; ++v) out_phi[v] = y[m * n + v] / s2[v];
  // constraint row (unscaled): sum w d_phi under crack control, d_E under strain control
  *out_E = yE;
  return RVE_OK;
}

// ---- checkpoint -----------------------------------------------------------------------------
static const char kMagic[8] = {'R', 'V', 'E', 'C', 'K', 'P', '0', '3'};

int rve_save(const rve_t *hc, const char *path) {
  rve *h = (rve *)hc;
  if (!h || !path) return RVE_E_ARG;
  const size_t n = h->g.n, m = h->m;
  std::vector<double> eps(m * n), phi(n), H(n);
  std::vector<uint8_t> mat(n);
  CK(cudaMemcpy(eps.data(), h->eps_c, 8 * m * n, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(phi.data(), h->phi_c, 8 * n, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(H.data(), h->Hn, 8 * n, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(mat.data(), h->mat, n, cudaMemcpyDeviceToHost));
  FILE *f = fopen(path, "wb");
  if (!f) {
    set_err(h, "cannot open %s", path);
    return RVE_E_IO;
  }
  bool ok = fwrite(kMagic, 1, 8, f) == 8;
  ok = ok && fwrite(&h->desc, sizeof h->desc, 1, f) == 1;
  int np = h->n_phases;
  ok = ok && fwrite(&np, sizeof np, 1, f) == 1;
  ok = ok && fwrite(h->E_ph.data(), 8, np, f) == (size_t)np;
  ok = ok && fwrite(h->nu_ph.data(), 8, np, f) == (size_t)np;
  ok = ok && fwrite(h->Gc_ph.data(), 8, np, f) == (size_t)np;
  ok = ok && fwrite(mat.data(), 1, n, f) == n;
  ok = ok && fwrite(eps.data(), 8, m * n, f) == m * n;
  ok = ok && fwrite(phi.data(), 8, n, f) == n;
  ok = ok && fwrite(H.data(), 8, n, f) == n;
  double sc[2] = {h->E_c, h->tau_c};
  ok = ok && fwrite(sc, 8, 2, f) == 2;
  int fl[8] = {h->started, h->notch_set, h->tuned, h->Px, h->Wy, h->pvar[0], h->pvar[1], h->pvar[2]};
  ok = ok && fwrite(fl, sizeof(int), 8, f) == 8;
  ok = (fclose(f) == 0) && ok;
  if (!ok) {
    set_err(h, "write to %s failed", path);
    return RVE_E_IO;
  }
  return RVE_OK;
}

int rve_load(const char *path, rve_t **out) {
  rve *h = nullptr;
  if (!path || !out) return RVE_E_ARG;
  *out = nullptr;
  FILE *f = fopen(path, "rb");
  if (!f) {
    set_err(nullptr, "cannot open %s", path);
    return RVE_E_IO;
  }
  char mg[8];
  rve_desc d;
  int np = 0;
  bool ok = fread(mg, 1, 8, f) == 8 && memcmp(mg, kMagic, 8) == 0;
  ok = ok && fread(&d, sizeof d, 1, f) == 1;
  ok = ok && fread(&np, sizeof np, 1, f) == 1 && np >= 1 && np <= RVE_MAX_PHASES;
  if (!ok) {
    fclose(f);
    set_err(nullptr, "%s is not an rve checkpoint", path);
    return RVE_E_IO;
  }
  std::vector<double> E(np), nu(np), Gc(np);
  ok = fread(E.data(), 8, np, f) == (size_t)np && fread(nu.data(), 8, np, f) == (size_t)np &&
       fread(Gc.data(), 8, np, f) == (size_t)np;
  const size_t n = (size_t)d.nx * d.ny * d.nz;
  const size_t m = d.nz == 1 ? 3 : 6;
  std::vector<uint8_t> mat(n), phase(n), mask(n);
  std::vector<double> eps(m * n), phi(n), H(n);
  double sc[2];
  int fl[8];
  ok = ok && fread(mat.data(), 1, n, f) == n && fread(eps.data(), 8, m * n, f) == m * n &&
       fread(phi.data(), 8, n, f) == n && fread(H.data(), 8, n, f) == n && fread(sc, 8, 2, f) == 2 &&
       fread(fl, sizeof(int), 8, f) == 8;
  fclose(f);
  if (!ok) {
    set_err(nullptr, "%s is truncated", path);
    return RVE_E_IO;
  }
  for (size_t v = 0; v < n; ++v) {
    phase[v] = mat[v] & 0x7f;
    mask[v] = (mat[v] & RVE_NOTCH_BIT) ? 1 : 0;
  }
  d.phase = phase.data();
  d.E = E.data();
  d.nu = nu.data();
  d.Gc = Gc.data();
  int rc = rve_create(&d, &h);
  if (rc != RVE_OK) return rc;
  if (fl[1]) rc = rve_set_notch(h, mask.data());
  if (rc == RVE_OK) rc = rve_set_state(h, eps.data(), phi.data(), H.data(), sc[0], sc[1]);
  if (rc != RVE_OK) {
    rve_destroy(h);
    return rc;
  }
  h->started = fl[0];
  if (fl[2]) {
    apply_tiles(h, fl[3], fl[4]);
    for (int a = 0; a < 3 && rc == RVE_OK; ++a)
      if (fl[5 + a] != h->pvar[a]) {
        if (fl[5 + a] < 0 || fl[5 + a] >= kPlanVariants) rc = RVE_E_IO;
        else rc = set_plan_variant(h, a, fl[5 + a]);
      }
    if (rc != RVE_OK) {
      rve_destroy(h);
      return rc;
    }
  }
  *out = h;
  return RVE_OK;
}

// Batched increments: every handle advances on its own stream (a non-blocking stream is
// created for handles still on the legacy default stream), driven by a pool of host
// threads, so the small, latency-bound FFT passes and reductions of different RVEs overlap
// on the device.  Each handle's arithmetic is independent of the others: results equal
// those of separate rve_crack_increment calls.  RVE_THREADS caps the pool size.
int rve_batch_crack_increment(rve_t **hs, int count, const double *da, rve_step *out, int *status) {
  if (!hs || count < 0 || !da) return RVE_E_ARG;
  for (int i = 0; i < count; ++i) {
    rve *h = hs[i];
    if (!h) continue;
    if (h->stream == 0) {
      cudaStream_t st;
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        set_err(h, "cudaStreamCreateWithFlags failed");
        return RVE_E_CUDA;
      }
      h->stream = st;
      h->own_stream = 1;
    }
  }
  // tune each distinct shape once, serially (timings taken under concurrency are noisy)
  if (autotune_enabled())
    for (int i = 0; i < count; ++i)
      if (hs[i] && !hs[i]->tuned) TRY(autotune(hs[i]));
  // RVEs of equal shape, precision and tiles share a KGroup: their Krylov chunks run as one
  // launch per pass (RVE_GROUP=0: every RVE on its own stream)
  std::vector<KGroup *> groups;
  {
    const char *ge = getenv("RVE_GROUP");
    if (!(ge && ge[0] == '0')) {
      std::map<std::vector<long long>, std::vector<rve *>> byk;
      for (int i = 0; i < count; ++i) {
        rve *h = hs[i];
        if (!h || h->kgroup) continue;
        byk[{h->g.nx, h->g.ny, h->g.nz, h->mixed, h->m, h->Px, h->Wy, h->Wz, h->Px_d, h->Wy_d, h->Wz_d, h->tr,
             h->pvar[0], h->pvar[1], h->pvar[2]}]
            .push_back(h);
      }
      for (auto &kv : byk) {
        // consecutive runs of group_max() members form one group each
        const int gm = group_max();
        for (size_t b = 0; b + 1 < kv.second.size(); b += gm) {
          KGroup *G = new KGroup();
          if (cudaStreamCreateWithFlags(&G->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete G;
            continue;
          }
          groups.push_back(G);
          for (size_t i = b; i < kv.second.size() && i < b + gm; ++i) kv.second[i]->kgroup = G;
        }
      }
    }
  }
  int nthreads = (int)std::thread::hardware_concurrency();
  const char *e = getenv("RVE_THREADS");
  if (e && atoi(e) > 0) nthreads = atoi(e);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > count) nthreads = count;
  std::vector<int> rcs(count, RVE_OK);
  // Longest expected increment first (list scheduling by decreasing cost): the threads take
  // the RVEs in this order, so the largest solves start at once instead of forming the tail
  // of the step.  Expected cost = operator applies of the RVE's last increment (a first
  // increment counts 600) x voxels x channels, scaled by 2 for float64; ties keep the caller's
  // order.  RVE_BATCH_ORDER=fifo keeps the caller's order throughout.
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  {
    const char *oe = getenv("RVE_BATCH_ORDER");
    if (!(oe && strcmp(oe, "fifo") == 0)) {
      std::vector<double> cost(count, 0.0);
      for (int i = 0; i < count; ++i) {
        const rve *h = hs[i];
        if (!h) continue;
        const double ap = h->last_applies > 0 ? (double)h->last_applies : 600.0;
        cost[i] = ap * (double)h->g.n * h->c * (h->mixed ? 1.0 : 2.0);
      }
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    }
  }
  std::atomic<int> next(0);
  int dev = 0;
  cudaGetDevice(&dev);
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= count) break;
      const int i = order[k];
      rcs[i] = hs[i] ? rve_crack_increment(hs[i], da[i], out ? &out[i] : nullptr) : RVE_E_ARG;
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t) pool.emplace_back(worker);
  for (auto &t : pool) t.join();
  for (int i = 0; i < count; ++i)
    if (hs[i]) hs[i]->kgroup = nullptr;
  for (KGroup *G : groups) {
    cudaStreamSynchronize(G->stream);
    cudaStreamDestroy(G->stream);
    delete G;
  }
  int first = RVE_OK;
  for (int i = 0; i < count; ++i) {
    if (status) status[i] = rcs[i];
    if (rcs[i] != RVE_OK && first == RVE_OK) first = rcs[i];
  }
  return first;
}

// ---- launch groups shared by handles that different host threads advance (the server) ----
// Handles of equal shape, precision and tiles join a KGroup of the pool for as long as they
// live (join after creation, leave before destruction), so their Krylov chunks run as grouped
// launches exactly as in rve_batch_crack_increment; groups hold up to group_max() members.
struct KGroupPool {
  std::mutex mu;
  std::map<std::vector<long long>, std::vector<std::pair<KGroup *, int>>> groups;
};

static std::vector<long long> group_key(const rve *h) {
  return {h->g.nx, h->g.ny, h->g.nz, h->mixed, h->m, h->Px, h->Wy, h->Wz, h->Px_d, h->Wy_d, h->Wz_d, h->tr,
          h->pvar[0], h->pvar[1], h->pvar[2]};
}

RVE_INTERNAL void *rve_group_pool_create() { return new KGroupPool(); }

RVE_INTERNAL void rve_group_pool_destroy(void *pp) {
  KGroupPool *pool = (KGroupPool *)pp;
  if (!pool) return;
  for (auto &kv : pool->groups)
    for (auto &g : kv.second) {
      cudaStreamSynchronize(g.first->stream);
      cudaStreamDestroy(g.first->stream);
      delete g.first;
    }
  delete pool;
}

RVE_INTERNAL int rve_group_pool_join(void *pp, rve_t *h) {
  KGroupPool *pool = (KGroupPool *)pp;
  if (!pool || !h || h->kgroup) return RVE_E_ARG;
  if (autotune_enabled() && !h->tuned) TRY(autotune(h));  // tiles are part of the key
  std::lock_guard<std::mutex> lk(pool->mu);
  auto &v = pool->groups[group_key(h)];
  for (auto &g : v)
    if (g.second < group_max()) {
      g.second += 1;
      h->kgroup = g.first;
      return RVE_OK;
    }
  KGroup *G = new KGroup();
  if (cudaStreamCreateWithFlags(&G->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete G;
    set_err(h, "cudaStreamCreateWithFlags failed");
    return RVE_E_CUDA;
  }
  v.emplace_back(G, 1);
  h->kgroup = G;
  return RVE_OK;
}

RVE_INTERNAL void rve_group_pool_leave(void *pp, rve_t *h) {
  KGroupPool *pool = (KGroupPool *)pp;
  if (!pool || !h || !h->kgroup) return;
  std::lock_guard<std::mutex> lk(pool->mu);
  auto it = pool->groups.find(group_key(h));
  if (it != pool->groups.end()) {
    auto &v = it->second;
    for (size_t i = 0; i < v.size(); ++i)
      if (v[i].first == h->kgroup) {
        if (--v[i].second == 0) {
          cudaStreamSynchronize(v[i].first->stream);
          cudaStreamDestroy(v[i].first->stream);
          delete v[i].first;
          v.erase(v.begin() + i);
        }
        break;
      }
  }
  h->kgroup = nullptr;
}

}  // extern "C"

// ================================ allocation-free apply =======================================
// rve_apply_device_noalloc: the scaled operator apply of rve_apply_device, with its spectral
// scratch and reduction partials taken from one file-scope device array instead of the
// buffers the handle allocated.  It exists for callers that may not allocate device memory
// at the time they call: code that runs while a CUDA graph is being captured (allocation is
// not a capturable operation), hosts whose device memory is owned by another allocator
// (e.g. a framework's caching pool) and that forbid the solver from growing it, and
// latency-bound service loops that pre-reserve everything at start-up.  The handle and the
// caller's input/output buffers must already exist; the call itself allocates nothing.
#include <mutex>

namespace {

// Largest scratch one call may use: spectral data (c * rows * hx complex values of the
// Krylov precision) plus the per-block reduction partials.  16 MiB + 256 KiB covers e.g. a
// 512 x 512 2D grid in float64 or a 64^3 3D grid in float32.  Every GPU that loads the
// library holds this array until the process exits.
constexpr size_t kNoAllocSpecBytes = 16u << 20;
constexpr size_t kNoAllocPartBytes = 256u << 10;
constexpr size_t kNoAllocBytes = kNoAllocSpecBytes + kNoAllocPartBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device, fetched once with that device current.
constexpr int kMaxDevices = 64;
static void *g_noalloc_ptr[kMaxDevices] = {};
static std::mutex g_noalloc_mu;

static int noalloc_setup(rve *h, void **out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_err(h, "device %d out of range for the allocation-free scratch", dev);
    return RVE_E_ARG;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return RVE_OK;
}

template <typename TK, int M>
static int apply_noalloc_t(rve *h, void *scratch, TK *x, const double *xE_ptr, TK *y) {
  // the handle's apply path, with the spectral scratch and the partials in the static array
  return apply_scaled<TK, M>(h, x, xE_ptr, y, 0, 0, nullptr, nullptr, nullptr, nullptr, nullptr,
                             (cpx<TK> *)scratch, (double *)((unsigned char *)scratch + kNoAllocSpecBytes));
}

}  // namespace

extern "C" int rve_apply_device_noalloc(rve_t *h, const void *x, const double *xE, void *y, double *yE) {
  if (!h || !x || !xE || !y || !yE) return RVE_E_ARG;
  if (!h->lin_valid) {
    set_err(h, "rve_apply_device_noalloc needs rve_linearize first");
    return RVE_E_STATE;
  }
  const size_t tk = h->mixed ? 4 : 8;
  const size_t spec = 2 * tk * (size_t)h->c * (size_t)h->g.rows * (size_t)h->g.hx;
  const int Gx = h->mixed ? h->Gx : h->Gx_d;
  const size_t part = 3 * sizeof(double) * (size_t)Gx;
  if (spec > kNoAllocSpecBytes || part > kNoAllocPartBytes) {
    set_err(h,
            "rve_apply_device_noalloc: this grid needs %zu bytes of spectral scratch and %zu of "
            "partials; the built-in array holds at most %zu and %zu",
            spec, part, kNoAllocSpecBytes, kNoAllocPartBytes);
    return RVE_E_ARG;
  }
  void *scratch = nullptr;
  TRY(noalloc_setup(h, &scratch));
  h->launches = 0;
  if (h->mixed) {
    if (h->m == 3) TRY((apply_noalloc_t<float, 3>(h, scratch, (float *)x, xE, (float *)y)));
    else TRY((apply_noalloc_t<float, 6>(h, scratch, (float *)x, xE, (float *)y)));
  } else {
    if (h->m == 3) TRY((apply_noalloc_t<double, 3>(h, scratch, (double *)x, xE, (double *)y)));
    else TRY((apply_noalloc_t<double, 6>(h, scratch, (double *)x, xE, (double *)y)));
  }
  if (h->lin_control == RVE_CTRL_STRAIN) {
    CK(cudaMemcpyAsync(yE, xE, sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  } else {
    const double *pd = (const double *)((unsigned char *)scratch + kNoAllocSpecBytes);
    k_reduce<<<1, 256, 0, h->stream>>>(pd, Gx, 1, 0, yE);
    h->launches += 1;
    CKL();
  }
  return RVE_OK;
}
