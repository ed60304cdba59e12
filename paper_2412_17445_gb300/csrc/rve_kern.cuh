// Kernel interface of librve: argument structs shared by the kernel files and the host
// driver, block reductions, and the per-voxel material byte encoding.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft.cuh"

#define RVE_NOTCH_BIT 0x80  // material byte: bit 7 = notch (phi held at 1), bits 0..6 = phase

// Phase property table (device constant memory, one table per RVE is passed by value).
struct PhaseTab {
  double lam[16], mu[16], Gc[16];
};

// Grid description.
struct Geo {
  int d, m, c;          // dimension, Mandel components, channels (m + 1)
  int nx, ny, nz;
  int hx;               // nx / 2 + 1 half-spectrum row length
  int rows;             // ny * nz real rows of length nx
  long long n;          // voxels
};

// Per-axis frequency tables (natural index k in [0, N)):
//   sn = sin(pi ks / N), cs = cos(pi ks / N) (exactly 0 at the Nyquist index), xi2 = (2 pi ks / N)^2
// with ks the signed wave number.
template <typename T>
struct AxisTab {
  const T *sn[3], *cs[3], *xi2[3];
};

// Tangent channels of the scaled Newton operator, per voxel (structure of arrays, stride n):
//   [0, NC)            C' = s1 * C_t in Mandel form, upper triangle row by row (NC = m(m+1)/2)
//   [NC, NC+m)         sF1 = s1 * g'(phi) sigma_drive
//   NC+m               kappa = chi * s2 / s1 (free voxels), 0 on the notch
//   NC+m+1             a' = s2 * (Gc/l + 2H) (free), 0 on the notch
//   NC+m+2             w = (phi/l + l L phi) (free), 0 on the notch
//   NC+m+3             b' = s2 * Gc * l (free), 0 on the notch
//   NC+m+4             notch indicator (1 on the notch, else 0)
template <int M>
struct TanIdx {
  static constexpr int NC = M * (M + 1) / 2;
  static constexpr int SF = NC;
  static constexpr int KAPPA = NC + M;
  static constexpr int A = NC + M + 1;
  static constexpr int W = NC + M + 2;
  static constexpr int B = NC + M + 3;
  static constexpr int NOTCH = NC + M + 4;
  static constexpr int K = NC + M + 5;
};

// Several fixed-order reductions of per-block partials in one single-block launch
// (k_reduce_list): segment i reduces NQ quantities of G partials each (sum, or max when
// is_max) into out[off + q].
struct ReduceSeg {
  const double *part;
  int G, NQ, is_max, off;
};
struct ReduceList {
  ReduceSeg s[4];
  int n;
};

// Device scalars of one BiCGStab solve (read by every Krylov kernel).
struct KrylovScalars {
  double rho, alpha, omega, beta;
  double bn2, atol2, tol2;
  double rn2;
  double s3;            // row scaling of the constraint row
  // E-slots (scalar component) of the Krylov vectors
  double xE, rE, rhE, pE, vE, sE, tE;
  double bE;            // E slot of the right-hand side (kept for restarts)
  double escale;        // column scaling of the E unknown in this solve
  int strain;           // 1: constraint row is d_E (strain control), else s3 sum w d_phi
  int done;             // 1 once converged / stopped
  int status;           // 0 converged, 1 iteration limit, 2 breakdown
  int iters;
  int maxit;
  int fault_rho0;       // fault injection: the finalisers see rho = 0 (a breakdown)
  int pending;          // float32 chunks: x += alpha p + omega s, r = s - omega t of the last
                        // iteration not applied yet (the next x-forward pass, or the chunk's
                        // closing k_kx_finish, applies it)
};

// ---- block reductions into per-block partials ------------------------------------------
// Sum NQ doubles over the block; thread 0 writes part[q * G + blk].
template <int NQ>
__device__ __forceinline__ void block_partials(double (&v)[NQ], double *part, int G, int blk) {
  __shared__ double red[32][NQ > 0 ? NQ : 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[wid][q] = x;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double x = lane < nw ? red[lane][q] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) part[q * G + blk] = x;
    }
  }
  __syncthreads();
}

// As block_partials for per-thread sums held in the Krylov precision TK: with TK = float the
// warp-level shuffle tree stays in float32 (32 terms) and only the per-warp sums are added in
// float64, which keeps the float64 pipe (1/64 of the float32 rate) out of the float32 passes.
template <typename TK, int NQ>
__device__ __forceinline__ void block_partials_k(const TK (&v)[NQ], double *part, int G, int blk) {
  if constexpr (sizeof(TK) == 8) {
    double w[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) w[q] = (double)v[q];
    block_partials<NQ>(w, part, G, blk);
  } else {
    __shared__ double red[32][NQ > 0 ? NQ : 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      float x = v[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) red[wid][q] = (double)x;
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
      const int nw = (blockDim.x + 31) >> 5;
      double sum = 0.0;
      for (int w = 0; w < nw; ++w) sum += red[w][threadIdx.x];
      part[threadIdx.x * G + blk] = sum;
    }
    __syncthreads();
  }
}

template <int NQ>
__device__ __forceinline__ void block_max_partials(double (&v)[NQ], double *part, int G, int blk) {
  __shared__ double red[32][NQ > 0 ? NQ : 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    if (lane == 0) red[wid][q] = x;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double x = lane < nw ? red[lane][q] : -1.0e308;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
      if (lane == 0) part[q * G + blk] = x;
    }
  }
  __syncthreads();
}

// ---- kernel argument structs ------------------------------------------------------------
// Operator apply: y = S J x (scaled Jacobian of the linearisation).
template <typename T>
struct ApplyArgs {
  Geo g;
  T *x;                 // c channels (written back when a fused update forms it)
  T *y;                 // c channels (phi channel also holds the pointwise part between passes)
  const T *tan;         // tangent channels (TanIdx)
  const double *xE_ptr; // E slot of x (device scalar)
  double e_scale;       // column scaling of the E unknown: d_E = e_scale * xE (ks == nullptr)
  double fM[6];         // load direction (Mandel)
  cpx<T> *spec;         // spectral scratch c * rows * hx
  double *part;         // per-block partials
  // fused BiCGStab vector updates (prologue) and dots (epilogue)
  int pro_mode;         // 0: x as given; 1: x := r + beta (x - omega v); 2: x := r - alpha v;
                        // 4: projection only (strain channels of x through G, nothing else);
                        // 5: as 1, after the pending update of the previous iteration
                        //    (xs += alpha x + omega s, r := s - omega t) when ks->pending
  T *r;                 // (written in mode 5)
  const T *v, *rhat, *s;  // operands of the fused updates / dots
  T *xs;                // mode 5: the Krylov solution vector
  const T *t;           // mode 5: A s of the previous iteration
  int epi_mode;         // 0: none; 1: dot(rhat, y); 2: dots (y, s), (y, y); 3: projection
                        // (writes the m strain channels of y only); 6: dots (y, s), (y, y),
                        // (rhat, s), (rhat, y), (s, s) for the merged omega / convergence update
  const KrylovScalars *ks;
  int tr;               // 1: spectral scratch transposed [ch][kx][row] (fused 2D column pass)
  // finalisation by the x-inverse pass itself (krylov_fin.cuh): 0 none; 1 / 2 the member's
  // last block runs the alpha / omega update on ksw (epilogue modes 1 / 2); 3 block 0 writes
  // yE = sum of the constraint-row partials; 4 block 0 copies *xE_ptr to yE (strain control);
  // 5 the last block runs the alpha update and clears ks->pending; 6 the last block runs the
  // merged omega / convergence update (epilogue mode 6) and sets ks->pending
  int fin;
  KrylovScalars *ksw;
  unsigned int *arrive; // arrival counter of the member (fin 1, 2)
  double *yE;           // fin 3, 4
};

// Residual: spectral data of (sigma, phi) in float64, epilogue forms F, rhs and w.
struct ResidArgs {
  Geo g;
  const double *sigma;  // m channels
  const double *phi;    // 1 channel
  const double *H;      // current history max(psi+, H^n)
  const uint8_t *mat;
  PhaseTab ph;
  double ell, s1, Lbar;
  cpx<double> *spec;
  double *F;            // unscaled residual F1 (m ch), F2 (1 ch)
  double *Lphi;         // L phi
  void *rhs;            // Krylov rhs b = -S F (krylov precision), c channels
  int rhs_double;       // 1 if rhs is double
  void *tan;            // tangent channels (w written here)
  int tan_double;
  int tanK;             // number of tangent channels
  double *part;
};

// Column (y / z) pass of the spectral data.
template <typename T>
struct ColArgs {
  Geo g;
  cpx<T> *spec;
  int axis;          // 1 = y, 2 = z
  int W;             // kx columns per block (a power of two)
  int lw;            // log2 W
  FftPlan plan;      // along the axis
  FftPlan yplan;     // y plan (3D z-pass: ky of a stored row is digit_reverse(yplan, y))
  AxisTab<T> tab;
  T inv_n;
  const KrylovScalars *ks;
};

// Constitutive update at one Newton iterate (float64).
struct ConstArgs {
  Geo g;
  const double *eps_t;  // m channels
  const double *phi;
  const double *Hn;
  const uint8_t *mat;
  PhaseTab ph;
  double fM[6];
  double E;
  double ell, k_res, s1, Lbar;
  int isotropic;
  double *sigma;        // m channels out
  double *H;            // max(psi+, H^n) out
  double *part;         // partials: m stress sums, |s1 sigma|^2
  double *part_max;     // partial max of 2 psi+ / (Gc / l) over free voxels
};

// Krylov vectors: c channels of n values (type TK); E slots live in KrylovScalars.
template <typename TK>
struct KvArgs {
  long long len;        // c * n
  int c;
  long long n;
  TK *x, *r, *rhat, *p, *v, *s, *t;
  KrylovScalars *ks;
  double *part;
  int G;
  unsigned int *arrive; // non-null: the last block of k_kxr runs the convergence test
};

// ---- groups: one launch over several RVEs of the same shape ----------------------------
// Passed by value as __grid_constant__ kernel parameters; member i is handled by the blocks
// with blockIdx.y == i (blockIdx.z for the 3D column passes, blockIdx.x for the
// single-block finalisers).  A solo launch is a group of one.
constexpr int kGroupMax = 8;

template <typename T>
struct ApplyGroup {
  ApplyArgs<T> m[kGroupMax];
};

template <typename T>
struct ColGroup {
  ColArgs<T> base;                       // geometry, plans, tables (shared by the members)
  cpx<T> *spec[kGroupMax];               // per member: spectral scratch
  const KrylovScalars *ks[kGroupMax];    // per member: Krylov scalars (or null)
};

template <typename TK>
struct KvGroup {
  KvArgs<TK> m[kGroupMax];
};

