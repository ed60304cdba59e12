// Residual FFT passes (Eq. System_CrackLength, float64) and the runtime-length
// instantiations of the apply passes (fft_passes.cuh).
#include "fft_passes.cuh"

// =========================== residual (float64) ==============================================
// x-forward of (sigma [m channels], phi [1 channel]).
template <int M>
__global__ void __launch_bounds__(256) k_xfwd_resid(ResidArgs a, FftPlan pl, int P) {
  extern __shared__ unsigned char smraw[];
  cpx<double> *sm = reinterpret_cast<cpx<double> *>(smraw);
  const Geo &g = a.g;
  const int c = M + 1, nx = g.nx, Np = pl.Np;
  const int n = (int)g.n;
  const int row0 = blockIdx.x * 2 * P;
  const int tot = 2 * P * nx;
  const FDiv dnx = make_fdiv(nx);
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int rr = (int)fdiv(i, dnx), x = i - rr * nx;
    const int row = row0 + rr;
    const int v = row * nx + x;
    const int l0 = rr >> 1;
    const int part = rr & 1;
    const int px = pad8(x);
#pragma unroll
    for (int k = 0; k <= M; ++k) {
      double val = 0;
      if (row < g.rows) val = (k < M) ? a.sigma[k * n + v] : a.phi[v];
      double *dst = reinterpret_cast<double *>(&sm[(k * P + l0) * Np + px]);
      dst[part] = val;
    }
  }
  xfwd_tail<double, 0>(sm, c, P, row0, g, pl, a.spec);
}

// x-inverse + residual epilogue: F1 = projected sigma, L phi, F2 (Eq. System_CrackLength),
// the Newton rhs b = -S F in the Krylov precision, w = d Gamma / d phi, and partials
//   0 Gamma_v = phi (phi/(2l) + (l/2) L phi)     1 w^2
//   2 |b_eps|^2     3 |b_phi|^2     4 reference magnitude of the F2 terms (squared)
template <int M, typename TK>
__global__ void __launch_bounds__(256) k_xinv_resid(ResidArgs a, FftPlan pl, int P, TK *rhs,
                                                    TK *tan, double *s2out) {
  extern __shared__ unsigned char smraw[];
  cpx<double> *sm = reinterpret_cast<cpx<double> *>(smraw);
  using TI = TanIdx<M>;
  const Geo &g = a.g;
  const int c = M + 1, nx = g.nx, Np = pl.Np;
  const int n = (int)g.n;
  const int row0 = blockIdx.x * 2 * P;
  const FDiv dnx = make_fdiv(nx);
  xinv_head<double, 0>(sm, c, P, row0, g, pl, a.spec);
  double acc[5] = {0, 0, 0, 0, 0};
  const int tot = 2 * P * nx;
  const double ell = a.ell;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int rr = (int)fdiv(i, dnx), x = i - rr * nx;
    const int row = row0 + rr;
    if (row >= g.rows) continue;
    const int v = row * nx + x;
    const int l0 = rr >> 1;
    const bool odd = rr & 1;
    const int px = pad8(x);
    double val[M + 1];
#pragma unroll
    for (int k = 0; k <= M; ++k) {
      const cpx<double> z = sm[(k * P + l0) * Np + px];
      val[k] = odd ? z.y : z.x;
    }
    const uint8_t mb = a.mat[v];
    const bool notch = (mb & RVE_NOTCH_BIT) != 0;
    const int ph = mb & 0x7f;
    const double Gc = a.ph.Gc[ph];
    const double phi = a.phi[v], H = a.H[v], Lp = val[M];
    const double aa = Gc / ell + 2.0 * H;
    const double F2 = notch ? (phi - 1.0) : (aa * phi + Gc * ell * Lp - 2.0 * H);
    const double w = notch ? 0.0 : (phi / ell + ell * Lp);
    const double s2 = notch ? 1.0 : 1.0 / (aa + Gc * ell * a.Lbar);
    double be = 0;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      a.F[k * n + v] = val[k];
      const double b = -a.s1 * val[k];
      rhs[k * n + v] = (TK)b;
      be += b * b;
    }
    a.F[M * n + v] = F2;
    a.Lphi[v] = Lp;
    const double bp = -s2 * F2;
    rhs[M * n + v] = (TK)bp;
    tan[TI::W * n + v] = (TK)w;
    s2out[v] = s2;
    acc[0] += phi * (phi / (2.0 * ell) + 0.5 * ell * Lp);
    acc[1] += w * w;
    acc[2] += be;
    acc[3] += bp * bp;
    if (!notch) {
      const double t1 = s2 * aa * phi, t2 = s2 * 2.0 * H, t3 = s2 * Gc * ell * Lp;
      acc[4] += t1 * t1 + t2 * t2 + t3 * t3;
    }
  }
  block_partials<5>(acc, a.part, gridDim.x, blockIdx.x);
}

// x-inverse of a projected strain field: eps = F^-1{ G : F{eps} } (channels 0..m-1; the
// extra channel of the residual layout is discarded).  Keeps eps_tilde in the compatible
// space: Newton corrections only ever act on compatible directions, so incompatible
// round-off carried in by a Krylov step would otherwise never be removed.
template <int M>
__global__ void __launch_bounds__(256) k_xinv_proj(ResidArgs a, FftPlan pl, int P, double *eps) {
  extern __shared__ unsigned char smraw[];
  cpx<double> *sm = reinterpret_cast<cpx<double> *>(smraw);
  const Geo &g = a.g;
  const int c = M + 1, nx = g.nx, Np = pl.Np;
  const int n = (int)g.n;
  const int row0 = blockIdx.x * 2 * P;
  const FDiv dnx = make_fdiv(nx);
  xinv_head<double, 0>(sm, c, P, row0, g, pl, a.spec);
  const int tot = 2 * P * nx;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int rr = (int)fdiv(i, dnx), x = i - rr * nx;
    const int row = row0 + rr;
    if (row >= g.rows) continue;
    const int v = row * nx + x;
    const bool odd = rr & 1;
    const int px = pad8(x);
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const cpx<double> z = sm[(k * P + (rr >> 1)) * Np + px];
      eps[k * n + v] = odd ? z.y : z.x;
    }
  }
}

// ---- explicit instantiations (runtime line length) ----------------------------------------
#define INST_APPLY(T, M)                                                        \
  template __global__ void k_xfwd_apply<T, M, 0, 0, -1>(const __grid_constant__ ApplyGroup<T>, FftPlan, int);   \
  template __global__ void k_xinv_apply<T, M, 0, 0, -1>(const __grid_constant__ ApplyGroup<T>, FftPlan, int);   \
  template __global__ void k_col<T, M, 0, 0>(const __grid_constant__ ColGroup<T>);                       \
  template __global__ void k_col<T, M, 1, 0>(const __grid_constant__ ColGroup<T>);                       \
  template __global__ void k_col<T, M, 2, 0>(const __grid_constant__ ColGroup<T>);
INST_APPLY(float, 3)
INST_APPLY(float, 6)
INST_APPLY(double, 3)
INST_APPLY(double, 6)
template __global__ void k_xinv_proj<3>(ResidArgs, FftPlan, int, double *);
template __global__ void k_xinv_proj<6>(ResidArgs, FftPlan, int, double *);
template __global__ void k_xfwd_resid<3>(ResidArgs, FftPlan, int);
template __global__ void k_xfwd_resid<6>(ResidArgs, FftPlan, int);
template __global__ void k_xinv_resid<3, float>(ResidArgs, FftPlan, int, float *, float *, double *);
template __global__ void k_xinv_resid<6, float>(ResidArgs, FftPlan, int, float *, float *, double *);
template __global__ void k_xinv_resid<3, double>(ResidArgs, FftPlan, int, double *, double *, double *);
template __global__ void k_xinv_resid<6, double>(ResidArgs, FftPlan, int, double *, double *, double *);
