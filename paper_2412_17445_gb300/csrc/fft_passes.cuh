#pragma once
// FFT pass kernels of the operator apply (Eq. CrackLength_linearization) and the helpers
// they share with the residual passes (Eq. System_CrackLength).
//
// Every pass kernel takes the line length of its own axis as the template parameter NL:
// NL > 0 is a compile-time length, so index arithmetic, loop trip counts and the stage
// sequence fold to constants; NL = 0 reads the length from the runtime plan.  Both run the
// same stage sequence.  Instantiated in kernels_fft.cu (NL = 0, plus the residual kernels)
// and kernels_fft_<N>.cu (one compile-time length each, compiled in parallel).
//
// Layout: real fields are channel-major [ch][z][y][x]; the spectral scratch holds half
// spectra [ch][z][y][kx] with hx = nx/2 + 1 (kx natural order).  In 3D the y-forward pass
// leaves ky in digit-reversed order, which is exactly the input order the y-inverse pass
// needs (see fft.cuh), so no permutation is ever applied to whole fields.
//
// Passes of one apply:
//   2D: x-forward (+prologue) -> y fused (forward, projection / Laplacian, inverse)
//       -> x-inverse (+epilogue)                                      3 kernels
//   3D: x-forward -> y-forward -> z fused -> y-inverse -> x-inverse   5 kernels
// Two real rows are transformed together as one complex row (z = a + i b) and separated
// by Hermitian symmetry, so every FFT in the x passes is a full-length complex FFT.
#include "rve_kern.cuh"
#include "krylov_fin.cuh"

namespace {

constexpr double kSqrt2 = 1.41421356237309504880;
constexpr double kInvSqrt2 = 0.70710678118654752440;

__device__ __forceinline__ FDiv make_fdiv(unsigned d) {
  FDiv f;
  f.d = d;
  f.m = d > 1 ? (0xFFFFFFFFu / d) + 1u : 0u;
  return f;
}

// ---- spectral multiply ------------------------------------------------------------------
// Galerkin projection of a Mandel tensor at one frequency (Eq. GFourier, symmetric reading):
//   (G : tau)_ij = (tau n)_i n_j + n_i (tau n)_j - (n . tau . n) n_i n_j
template <typename T, int M>
__device__ __forceinline__ void project_mandel(T *t, const T *n, T scale) {
  if (M == 3) {
    const T txy = t[2] * (T)kInvSqrt2;
    const T v0 = t[0] * n[0] + txy * n[1];
    const T v1 = txy * n[0] + t[1] * n[1];
    const T s = n[0] * v0 + n[1] * v1;
    t[0] = scale * (2 * v0 * n[0] - s * n[0] * n[0]);
    t[1] = scale * (2 * v1 * n[1] - s * n[1] * n[1]);
    t[2] = scale * (T)kSqrt2 * (v0 * n[1] + n[0] * v1 - s * n[0] * n[1]);
  } else {
    const T txy = t[5] * (T)kInvSqrt2, txz = t[4] * (T)kInvSqrt2, tyz = t[3] * (T)kInvSqrt2;
    const T v0 = t[0] * n[0] + txy * n[1] + txz * n[2];
    const T v1 = txy * n[0] + t[1] * n[1] + tyz * n[2];
    const T v2 = txz * n[0] + tyz * n[1] + t[2] * n[2];
    const T s = n[0] * v0 + n[1] * v1 + n[2] * v2;
    t[0] = scale * (2 * v0 * n[0] - s * n[0] * n[0]);
    t[1] = scale * (2 * v1 * n[1] - s * n[1] * n[1]);
    t[2] = scale * (2 * v2 * n[2] - s * n[2] * n[2]);
    t[3] = scale * (T)kSqrt2 * (v1 * n[2] + n[1] * v2 - s * n[1] * n[2]);
    t[4] = scale * (T)kSqrt2 * (v0 * n[2] + n[0] * v2 - s * n[0] * n[2]);
    t[5] = scale * (T)kSqrt2 * (v0 * n[1] + n[0] * v1 - s * n[0] * n[1]);
  }
}

// Unit direction of the rotated-scheme modified frequency (Willot), 0 where it vanishes.
template <typename T, int D>
__device__ __forceinline__ void willot_n(const AxisTab<T> &tb, const int *k, T *n, T &xi2) {
  T sn[3], cs[3];
  xi2 = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    sn[a] = tb.sn[a][k[a]];
    cs[a] = tb.cs[a][k[a]];
    xi2 += tb.xi2[a][k[a]];
  }
  T nn = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    T v = sn[a];
#pragma unroll
    for (int b = 0; b < D; ++b)
      if (b != a) v *= cs[b];
    n[a] = v;
    nn += v * v;
  }
  if (nn > (T)0) {
    T inv = (T)1 / sqrt(nn);
#pragma unroll
    for (int a = 0; a < D; ++a) n[a] *= inv;
  } else {
#pragma unroll
    for (int a = 0; a < D; ++a) n[a] = 0;
  }
}

// ---- x-forward tail: DIF over the packed row pairs, then Hermitian unpack + store -------
// tr = 0: half spectra stored row-major [ch][row][kx] (coalesced along kx);
// tr = 1: stored transposed [ch][kx][row] for the fused 2D column pass (k_col_fused2d).
// With tr the threads walk the digit-reversed positions of each line (conflict-free shared
// reads; the partner N - k of position p lies at a nearly contiguous position) and write
// the two rows of a pair as one 16-byte store.
template <typename T, int NL>
__device__ __forceinline__ void xfwd_tail(cpx<T> *sm, int c, int P, int row0, const Geo &g, const FftPlan &pl,
                          cpx<T> *spec, int tr = 0) {
  const int nx = NL > 0 ? NL : g.nx, hx = nx / 2 + 1, Np = line_slots<NL>(pl.Np);
  __syncthreads();
  if constexpr (NL > 0) {
    fft_dif_ct<T, NL, 0>(sm, c * P, 0, (const cpx<T> *)pl.tw);
  } else {
    LineLayout ly;
    ly.L = c * P;
    ly.lw = 1;
    ly.lsA = Np;
    ly.lsB = 0;
    ly.es = 1;
    ly.line_fastest = false;
    fft_dif<T>(sm, ly, pl, (T)-1);
  }
  const int cs = g.rows * hx;
  const FDiv dhx = make_fdiv(hx), dP = make_fdiv(P);
  if (tr) {
    const int totp = c * P * nx;
    const FDiv dnx = make_fdiv(nx);
    for (int i = threadIdx.x; i < totp; i += blockDim.x) {
      const int l = NL > 0 ? i / NL : (int)fdiv(i, dnx);
      const int p = i - l * nx;
      int k;
      if constexpr (NL > 0) k = digit_rev_ct<NL>(p);
      else k = pl.rev[p];
      if (2 * k > nx) continue;
      const int kn = k == 0 ? 0 : nx - k;
      int pn;
      if constexpr (NL > 0) pn = digit_unrev_ct<NL>(kn);
      else pn = pl.unrev[kn];
      const int ch = (int)fdiv(l, dP), pr = l - ch * P;
      const cpx<T> zk = sm[l * Np + smap<NL>(p)];
      const cpx<T> zn = sm[l * Np + smap<NL>(pn)];
      const cpx<T> A = {(zk.x + zn.x) * (T)0.5, (zk.y - zn.y) * (T)0.5};
      const cpx<T> B = {(zk.y + zn.y) * (T)0.5, (zn.x - zk.x) * (T)0.5};
      const int r0 = row0 + 2 * pr;
      cpx<T> *dst = spec + ch * cs + k * g.rows + r0;
      if (r0 + 1 < g.rows) {
        if constexpr (sizeof(T) == 4) {
          *reinterpret_cast<float4 *>(dst) = make_float4(A.x, A.y, B.x, B.y);
        } else {
          dst[0] = A;
          dst[1] = B;
        }
      } else if (r0 < g.rows) {
        dst[0] = A;
      }
    }
    return;
  }
  const int tot = c * P * hx;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int l = NL > 0 ? i / (NL / 2 + 1) : (int)fdiv(i, dhx);
    const int k = i - l * hx;
    const int ch = (int)fdiv(l, dP), pr = l - ch * P;
    const cpx<T> zk = sm[l * Np + smap<NL>(pl.unrev[k])];
    const cpx<T> zn = sm[l * Np + smap<NL>(pl.unrev[k == 0 ? 0 : nx - k])];
    const cpx<T> A = {(zk.x + zn.x) * (T)0.5, (zk.y - zn.y) * (T)0.5};
    const cpx<T> B = {(zk.y + zn.y) * (T)0.5, (zn.x - zk.x) * (T)0.5};
    const int r0 = row0 + 2 * pr, r1 = r0 + 1;
    if (r0 < g.rows) spec[ch * cs + r0 * hx + k] = A;
    if (r1 < g.rows) spec[ch * cs + r1 * hx + k] = B;
  }
}

// ---- x-inverse head: load row pairs of half spectra, rebuild full lines, DIT inverse ----
template <typename T, int NL>
__device__ __forceinline__ void xinv_head(cpx<T> *sm, int c, int P, int row0, const Geo &g, const FftPlan &pl,
                          const cpx<T> *spec, int tr = 0) {
  const int nx = NL > 0 ? NL : g.nx, hx = nx / 2 + 1, Np = line_slots<NL>(pl.Np);
  const int cs = g.rows * hx;
  const int tot = c * P * hx;
  const FDiv dhx = make_fdiv(hx), dP = make_fdiv(P);
  if (tr) {
    // Z_k = A + iB for k <= nx/2 and Z_{nx-k} = conj(A) + i conj(B), with (A, B) the half-
    // spectrum entries of the row pair at k.  Threads walk the positions p of each line
    // (k = rev(p)); a position with k <= nx/2 loads its entry once and writes both p and the
    // partner position of nx - k.  All loads of a batch of U positions per thread are issued
    // before the first shared-memory write.
    const int totp = c * P * nx;
    const FDiv dnx = make_fdiv(nx);
    constexpr int U = 8;
    for (int base = 0; base < totp; base += U * (int)blockDim.x) {
      cpx<T> qa[U], qb[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = base + u * (int)blockDim.x + (int)threadIdx.x;
        qa[u] = {0, 0};
        qb[u] = {0, 0};
        if (i >= totp) continue;
        const int l = NL > 0 ? i / NL : (int)fdiv(i, dnx);
        const int p = i - l * nx;
        int k;
        if constexpr (NL > 0) k = digit_rev_ct<NL>(p);
        else k = pl.rev[p];
        if (2 * k > nx) continue;
        const int ch = (int)fdiv(l, dP), pr = l - ch * P;
        const int r0 = row0 + 2 * pr;
        const cpx<T> *src = spec + ch * cs + k * g.rows + r0;
        if (r0 + 1 < g.rows) {
          if constexpr (sizeof(T) == 4) {
            const float4 q = *reinterpret_cast<const float4 *>(src);
            qa[u] = {q.x, q.y};
            qb[u] = {q.z, q.w};
          } else {
            qa[u] = src[0];
            qb[u] = src[1];
          }
        } else if (r0 < g.rows) {
          qa[u] = src[0];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = base + u * (int)blockDim.x + (int)threadIdx.x;
        if (i >= totp) continue;
        const int l = NL > 0 ? i / NL : (int)fdiv(i, dnx);
        const int p = i - l * nx;
        int k;
        if constexpr (NL > 0) k = digit_rev_ct<NL>(p);
        else k = pl.rev[p];
        if (2 * k > nx) continue;
        cpx<T> A = qa[u], B = qb[u];
        if (k == 0 || 2 * k == nx) {
          A.y = 0;
          B.y = 0;
        }
        sm[l * Np + smap<NL>(p)] = cpx<T>{A.x - B.y, A.y + B.x};
        if (k > 0 && 2 * k < nx) {
          int pn;
          if constexpr (NL > 0) pn = digit_unrev_ct<NL>(nx - k);
          else pn = pl.unrev[nx - k];
          sm[l * Np + smap<NL>(pn)] = cpx<T>{A.x + B.y, B.x - A.y};
        }
      }
    }
  }
  for (int i = threadIdx.x; i < (tr ? 0 : tot); i += blockDim.x) {
    const int l = NL > 0 ? i / (NL / 2 + 1) : (int)fdiv(i, dhx);
    const int k = i - l * hx;
    const int ch = (int)fdiv(l, dP), pr = l - ch * P;
    const int r0 = row0 + 2 * pr, r1 = r0 + 1;
    cpx<T> A = {0, 0}, B = {0, 0};
    if (r0 < g.rows) A = spec[ch * cs + r0 * hx + k];
    if (r1 < g.rows) B = spec[ch * cs + r1 * hx + k];
    if (k == 0 || 2 * k == nx) {
      A.y = 0;
      B.y = 0;
    }
    sm[l * Np + smap<NL>(pl.unrev[k])] = {A.x - B.y, A.y + B.x};
    if (k > 0 && 2 * k < nx) sm[l * Np + smap<NL>(pl.unrev[nx - k])] = {A.x + B.y, B.x - A.y};
  }
  __syncthreads();
  if constexpr (NL > 0) {
    fft_dit_ct<T, NL, 0>(sm, c * P, 0, (const cpx<T> *)pl.tw);
  } else {
    LineLayout ly;
    ly.L = c * P;
    ly.lw = 1;
    ly.lsA = Np;
    ly.lsB = 0;
    ly.es = 1;
    ly.line_fastest = false;
    fft_dit<T>(sm, ly, pl, (T)1);
  }
}

}  // namespace

// =========================== operator apply ==================================================
// Prologue (per voxel): input dq = (d_eps, d_phi, dE) (optionally formed by a fused
// BiCGStab update), d_eps' = d_eps + f dE, d_phi masked on the notch;
//   t      = C' d_eps' + sF d_phi        (channels 0..m-1 of the FFT, row-scaled F1 input)
//   d_phi                                  (channel m of the FFT)
//   pw     = kappa (sF . d_eps') + a' d_phi + notch * dq_phi   (pointwise part of row F2)
//   sum w d_phi                            (constraint row, block partial 0)
// A thread takes the two voxels (x, r0) and (x, r0 + 1) of a row pair: all loads of both are
// issued before either is used, and the pair fills one complex shared-memory slot.
template <typename T, int M>
struct ProIn {
  T q[M + 1];                 // input vector (after the fused update)
  T cc[M * (M + 1) / 2];      // C' upper triangle
  T sF[M];
  T kappa, av, w, notch;
};

template <typename T, int M>
__device__ __forceinline__ void pro_load(const ApplyArgs<T> &a, int n, int v, T beta, T omega, T alpha,
                                         ProIn<T, M> &in, int pm, bool pending) {
  using TI = TanIdx<M>;
#pragma unroll
  for (int k = 0; k <= M; ++k) {
    const int o = k * n + v;
    T val;
    if (pm == 1) {
      val = a.r[o] + beta * (a.x[o] - omega * a.v[o]);
      a.x[o] = val;
    } else if (pm == 5) {
      // the previous iteration's x += alpha p + omega s, r = s - omega t (when pending), then
      // p := r + beta (p - omega v); omega and alpha are still the previous iteration's
      const T p = a.x[o];
      T r;
      if (pending) {
        const T sv = a.s[o];
        r = sv - omega * a.t[o];
        a.xs[o] += alpha * p + omega * sv;
        a.r[o] = r;
      } else {
        r = a.r[o];
      }
      val = r + beta * (p - omega * a.v[o]);
      a.x[o] = val;
    } else if (pm == 2) {
      val = a.r[o] - alpha * a.v[o];
      a.x[o] = val;
    } else {
      val = a.x[o];
    }
    in.q[k] = val;
  }
#pragma unroll
  for (int k = 0; k < TI::NC; ++k) in.cc[k] = a.tan[k * n + v];
#pragma unroll
  for (int k = 0; k < M; ++k) in.sF[k] = a.tan[(TI::SF + k) * n + v];
  in.kappa = a.tan[TI::KAPPA * n + v];
  in.av = a.tan[TI::A * n + v];
  in.w = a.tan[TI::W * n + v];
  in.notch = a.tan[TI::NOTCH * n + v];
}

template <typename T, int M>
__device__ __forceinline__ void pro_compute(const ApplyArgs<T> &a, int n, int v, const T (&fx)[M],
                                            const ProIn<T, M> &in, T (&out)[M + 1], T &wdp) {
  T de[M];
#pragma unroll
  for (int k = 0; k < M; ++k) de[k] = in.q[k] + fx[k];
  const T dpm = in.q[M] * ((T)1 - in.notch);
  T sde = 0;
#pragma unroll
  for (int k = 0; k < M; ++k) sde += in.sF[k] * de[k];
#pragma unroll
  for (int k = 0; k <= M; ++k) out[k] = 0;
  int idx = 0;
#pragma unroll
  for (int i2 = 0; i2 < M; ++i2) {
#pragma unroll
    for (int j2 = i2; j2 < M; ++j2) {
      const T cij = in.cc[idx];
      out[i2] += cij * de[j2];
      if (j2 != i2) out[j2] += cij * de[i2];
      ++idx;
    }
  }
#pragma unroll
  for (int k = 0; k < M; ++k) out[k] += in.sF[k] * dpm;
  out[M] = dpm;
  a.y[M * n + v] = in.kappa * sde + in.av * dpm + in.notch * in.q[M];
  wdp += in.w * dpm;
}

// float32: at least 4 resident blocks per SM (64 registers per thread)
#ifndef XFWD_MIN_BLOCKS_F32
#define XFWD_MIN_BLOCKS_F32 4
#endif
// PC > 0 / MODE >= 0: row pairs per block and prologue mode fixed at compile time (the
// float32 2D passes of the Krylov chunks), so every loop bound and branch folds; PC = 0 /
// MODE = -1 read them from the launch.
template <typename T, int M, int NL, int PC, int MODE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? XFWD_MIN_BLOCKS_F32 : 1) k_xfwd_apply(const __grid_constant__ ApplyGroup<T> grp, FftPlan pl, int P_rt) {
  const ApplyArgs<T> &a = grp.m[blockIdx.y];
  const int P = PC > 0 ? PC : P_rt;
  const int pm = MODE >= 0 ? MODE : a.pro_mode;
  extern __shared__ unsigned char smraw[];
  cpx<T> *sm = reinterpret_cast<cpx<T> *>(smraw);
  if (a.ks && a.ks->done) return;
  const Geo &g = a.g;
  const int c = M + 1, nx = NL > 0 ? NL : g.nx, Np = line_slots<NL>(pl.Np);
  const int n = (int)g.n;
  const int row0 = blockIdx.x * 2 * P;
  const FDiv dnx = make_fdiv(nx);
  const double xE = *a.xE_ptr * (a.ks ? a.ks->escale : a.e_scale);
  T fx[M];
#pragma unroll
  for (int k = 0; k < M; ++k) fx[k] = (T)a.fM[k] * (T)xE;
  T beta = 0, omega = 0, alpha = 0;
  bool pending = false;
  if (pm == 1) {
    beta = (T)a.ks->beta;
    omega = (T)a.ks->omega;
  } else if (pm == 5) {
    beta = (T)a.ks->beta;
    omega = (T)a.ks->omega;
    alpha = (T)a.ks->alpha;
    pending = a.ks->pending != 0;
  } else if (pm == 2) {
    alpha = (T)a.ks->alpha;
  }
  // per-thread and warp sums stay in T (a few dozen terms); the block and grid sums are float64
  T wdp = 0;
  const int tot = P * nx;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int l0 = NL > 0 ? i / NL : (int)fdiv(i, dnx), x = i - l0 * nx;
    const int r0 = row0 + 2 * l0;
    const bool ok0 = r0 < g.rows, ok1 = r0 + 1 < g.rows;
    const int v0 = r0 * nx + x, v1 = v0 + nx;
    T out0[M + 1], out1[M + 1];
#pragma unroll
    for (int k = 0; k <= M; ++k) out0[k] = out1[k] = 0;
    if (pm == 4) {
      // projection of the strain channels of x alone (Newton update direction)
#pragma unroll
      for (int k = 0; k < M; ++k) {
        if (ok0) out0[k] = a.x[k * n + v0];
        if (ok1) out1[k] = a.x[k * n + v1];
      }
    } else {
      if constexpr (M == 6) {
        // 3D: 38 operands per voxel; holding both voxels' operands at once spills at the 64
        // registers of four resident blocks, so the two voxels are loaded and used in turn
        ProIn<T, M> in;
        if (ok0) {
          pro_load<T, M>(a, n, v0, beta, omega, alpha, in, pm, pending);
          pro_compute<T, M>(a, n, v0, fx, in, out0, wdp);
        }
        if (ok1) {
          pro_load<T, M>(a, n, v1, beta, omega, alpha, in, pm, pending);
          pro_compute<T, M>(a, n, v1, fx, in, out1, wdp);
        }
      } else {
        ProIn<T, M> in0, in1;
        if (ok0) pro_load<T, M>(a, n, v0, beta, omega, alpha, in0, pm, pending);
        if (ok1) pro_load<T, M>(a, n, v1, beta, omega, alpha, in1, pm, pending);
        if (ok0) pro_compute<T, M>(a, n, v0, fx, in0, out0, wdp);
        if (ok1) pro_compute<T, M>(a, n, v1, fx, in1, out1, wdp);
      }
    }
    const int px = smap<NL>(x);
#pragma unroll
    for (int k = 0; k <= M; ++k) sm[(k * P + l0) * Np + px] = {out0[k], out1[k]};
  }
  const T pv[1] = {wdp};
  block_partials_k<T, 1>(pv, a.part, gridDim.x, blockIdx.x);
  xfwd_tail<T, NL>(sm, c, P, row0, g, pl, a.spec, a.tr);
}

// Epilogue (per voxel): y_eps = projected t (row scaling and 1/n folded in earlier),
// y_phi = pw + b' L d_phi; optional fused BiCGStab dots (block partials 1.. ).  A thread
// takes the two voxels of a row pair (one complex shared-memory slot per channel).
template <typename T, int M>
struct EpiIn {
  T pw, bb;
  T o[M + 1];   // rhat (mode 1) or s (modes 2, 6)
  T o2[M + 1];  // rhat (mode 6)
};

template <typename T, int M>
__device__ __forceinline__ void epi_load(const ApplyArgs<T> &a, int n, int v, EpiIn<T, M> &in, int em) {
  using TI = TanIdx<M>;
  if (em == 3) return;  // projection: strain channels only
  in.pw = a.y[M * n + v];
  in.bb = a.tan[TI::B * n + v];
  if (em == 1) {
#pragma unroll
    for (int k = 0; k <= M; ++k) in.o[k] = a.rhat[k * n + v];
  } else if (em == 2) {
#pragma unroll
    for (int k = 0; k <= M; ++k) in.o[k] = a.s[k * n + v];
  } else if (em == 6) {
#pragma unroll
    for (int k = 0; k <= M; ++k) {
      in.o[k] = a.s[k * n + v];
      in.o2[k] = a.rhat[k * n + v];
    }
  }
}

template <typename T, int M>
__device__ __forceinline__ void epi_compute(const ApplyArgs<T> &a, int n, int v, T (&yv)[M + 1],
                                            const EpiIn<T, M> &in, T (&d)[5], int em) {
  if (em == 3) {
#pragma unroll
    for (int k = 0; k < M; ++k) a.y[k * n + v] = yv[k];
    return;
  }
  yv[M] = in.pw + in.bb * yv[M];
#pragma unroll
  for (int k = 0; k <= M; ++k) a.y[k * n + v] = yv[k];
  if (em == 1) {
#pragma unroll
    for (int k = 0; k <= M; ++k) d[0] += in.o[k] * yv[k];
  } else if (em == 2) {
#pragma unroll
    for (int k = 0; k <= M; ++k) {
      d[0] += yv[k] * in.o[k];
      d[1] += yv[k] * yv[k];
    }
  } else if (em == 6) {
#pragma unroll
    for (int k = 0; k <= M; ++k) {
      d[0] += yv[k] * in.o[k];      // (t, s)
      d[1] += yv[k] * yv[k];        // (t, t)
      d[2] += in.o2[k] * in.o[k];   // (rhat, s)
      d[3] += in.o2[k] * yv[k];     // (rhat, t)
      d[4] += in.o[k] * in.o[k];    // (s, s)
    }
  }
}

template <typename T, int M, int NL, int PC, int MODE>
__global__ void __launch_bounds__(256) k_xinv_apply(const __grid_constant__ ApplyGroup<T> grp, FftPlan pl, int P_rt) {
  const ApplyArgs<T> &a = grp.m[blockIdx.y];
  const int P = PC > 0 ? PC : P_rt;
  const int em = MODE >= 0 ? MODE : a.epi_mode;
  extern __shared__ unsigned char smraw[];
  cpx<T> *sm = reinterpret_cast<cpx<T> *>(smraw);
  if (a.ks && a.ks->done) return;
  const Geo &g = a.g;
  const int c = M + 1, nx = NL > 0 ? NL : g.nx, Np = line_slots<NL>(pl.Np);
  const int n = (int)g.n;
  const int row0 = blockIdx.x * 2 * P;
  const FDiv dnx = make_fdiv(nx);
  xinv_head<T, NL>(sm, c, P, row0, g, pl, a.spec, a.tr);
  T d[5] = {0, 0, 0, 0, 0};  // per-thread and warp sums in T, block and grid sums in float64
  const int tot = P * nx;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int l0 = NL > 0 ? i / NL : (int)fdiv(i, dnx), x = i - l0 * nx;
    const int r0 = row0 + 2 * l0;
    const bool ok0 = r0 < g.rows, ok1 = r0 + 1 < g.rows;
    const int v0 = r0 * nx + x, v1 = v0 + nx;
    EpiIn<T, M> in0, in1;
    if (ok0) epi_load<T, M>(a, n, v0, in0, em);
    if (ok1) epi_load<T, M>(a, n, v1, in1, em);
    const int px = smap<NL>(x);
    T y0[M + 1], y1[M + 1];
#pragma unroll
    for (int k = 0; k <= M; ++k) {
      const cpx<T> z = sm[(k * P + l0) * Np + px];
      y0[k] = z.x;
      y1[k] = z.y;
    }
    if (ok0) epi_compute<T, M>(a, n, v0, y0, in0, d, em);
    if (ok1) epi_compute<T, M>(a, n, v1, y1, in1, d, em);
  }
  if (em == 6) {
    block_partials_k<T, 5>(d, a.part + gridDim.x, gridDim.x, blockIdx.x);
  } else if (em != 0) {
    const T pv[2] = {d[0], d[1]};
    block_partials_k<T, 2>(pv, a.part + gridDim.x, gridDim.x, blockIdx.x);
  }
  if (a.fin == 1 || a.fin == 2 || a.fin == 5 || a.fin == 6) {
    // the member's last block finalises the iteration's scalars (no separate launch)
    if (last_block_arrives(a.arrive, gridDim.x)) {
      if (a.fin == 1) fin_alpha<true>(a.ksw, a.part, gridDim.x);
      else if (a.fin == 2) fin_omega<true>(a.ksw, a.part, gridDim.x);
      else if (a.fin == 5) fin_alpha_clear<true>(a.ksw, a.part, gridDim.x);
      else fin_omega_conv<true>(a.ksw, a.part, gridDim.x);
    }
  } else if (a.fin == 3 && blockIdx.x == 0) {
    // the constraint-row partials come from the x-forward pass (an earlier launch)
    const double sE = sum_partials_t<false>(a.part, gridDim.x);
    if (threadIdx.x == 0) *a.yE = sE;
  } else if (a.fin == 4 && blockIdx.x == 0 && threadIdx.x == 0) {
    *a.yE = *a.xE_ptr;
  }
}

// =========================== column passes (y, z) ============================================

// MODE 0: forward only (DIF, result stays digit-reversed along the axis)
// MODE 1: forward, spectral multiply, inverse (the last axis)
// MODE 2: inverse only (input digit-reversed along the axis, DIT)
template <typename T, int M, int MODE, int NL>
__global__ void __launch_bounds__(256) k_col(const __grid_constant__ ColGroup<T> grp) {
  const ColArgs<T> &a = grp.base;
  cpx<T> *const spec = grp.spec[blockIdx.z];
  const KrylovScalars *const ks = grp.ks[blockIdx.z];
  extern __shared__ unsigned char smraw[];
  cpx<T> *sm = reinterpret_cast<cpx<T> *>(smraw);
  if (ks && ks->done) return;
  const Geo &g = a.g;
  const int c = M + 1;
  const int W = a.W, lw = a.lw;
  const int N = NL > 0 ? NL : a.plan.N, Np = line_slots<NL>(a.plan.Np);
  const int kx0 = blockIdx.x * W;
  const int other = blockIdx.y;
  int es_g, base_o;
  if (a.axis == 1) {
    es_g = g.hx;
    base_o = other * g.ny * g.hx;
  } else {
    es_g = g.hx * g.ny;
    base_o = other * g.hx;
  }
  const int cs = g.rows * g.hx;
  const int tot = (c * N) << lw;
  const FDiv dN = make_fdiv(N);
  // the block's lines are strided in the scratch (one L2 round trip per element): each thread
  // issues KU loads before its first shared-memory store, so they are in flight together
  constexpr int KU = 4;
  for (int base = 0; base < tot; base += KU * (int)blockDim.x) {
    cpx<T> val[KU];
    int slot[KU];
#pragma unroll
    for (int u = 0; u < KU; ++u) {
      const int i = base + u * (int)blockDim.x + (int)threadIdx.x;
      val[u] = {0, 0};
      slot[u] = -1;
      if (i < tot) {
        const int iw = i >> lw;
        const int w = i & (W - 1);
        const int ch = NL > 0 ? iw / NL : (int)fdiv(iw, dN);
        const int e = iw - ch * N;
        if (kx0 + w < g.hx) val[u] = spec[ch * cs + base_o + e * es_g + kx0 + w];
        slot[u] = ((ch * Np + smap<NL>(e)) << lw) + w;
      }
    }
#pragma unroll
    for (int u = 0; u < KU; ++u)
      if (slot[u] >= 0) sm[slot[u]] = val[u];
  }
  __syncthreads();
  LineLayout ly;
  ly.L = c * W;
  ly.dL = make_fdiv(c * W);
  ly.lw = W;
  ly.dlw = make_fdiv(W);
  ly.lsA = Np * W;
  ly.lsB = 1;
  ly.es = W;
  // W > 1: consecutive threads take consecutive columns (contiguous addresses); W = 1: the
  // lines (channels) are Np apart, a multiple of the bank count for power-of-two N, so
  // consecutive threads take consecutive butterflies of one line instead
  ly.line_fastest = W > 1;
  const cpx<T> *tw = (const cpx<T> *)a.plan.tw;
  if (MODE == 0 || MODE == 1) {
    if constexpr (NL > 0) fft_dif_ct<T, NL, -1>(sm, c, lw, tw);
    else fft_dif<T>(sm, ly, a.plan, (T)-1);
  }
  if (MODE == 1) {
    constexpr int D = (M == 3) ? 2 : 3;
    const int ky_other = (D == 3) ? a.yplan.rev[other] : 0;
    for (int i = threadIdx.x; i < (N << lw); i += blockDim.x) {
      const int p = i >> lw;
      const int w = i & (W - 1);
      if (kx0 + w >= g.hx) continue;
      int k[3];
      k[0] = kx0 + w;
      if (D == 2) {
        k[1] = a.plan.rev[p];
      } else {
        k[1] = ky_other;
        k[2] = a.plan.rev[p];
      }
      T nv[3], xi2;
      willot_n<T, D>(a.tab, k, nv, xi2);
      const int pp = smap<NL>(p);
      T re[M], im[M];
#pragma unroll
      for (int ch = 0; ch < M; ++ch) {
        const cpx<T> z = sm[((ch * Np + pp) << lw) + w];
        re[ch] = z.x;
        im[ch] = z.y;
      }
      project_mandel<T, M>(re, nv, a.inv_n);
      project_mandel<T, M>(im, nv, a.inv_n);
#pragma unroll
      for (int ch = 0; ch < M; ++ch) sm[((ch * Np + pp) << lw) + w] = {re[ch], im[ch]};
      cpx<T> zp = sm[((M * Np + pp) << lw) + w];
      const T sc = xi2 * a.inv_n;
      sm[((M * Np + pp) << lw) + w] = {zp.x * sc, zp.y * sc};
    }
    __syncthreads();
  }
  if (MODE == 1 || MODE == 2) {
    if constexpr (NL > 0) fft_dit_ct<T, NL, -1>(sm, c, lw, tw);
    else fft_dit<T>(sm, ly, a.plan, (T)1);
  }
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int iw = i >> lw;
    const int w = i & (W - 1);
    const int ch = NL > 0 ? iw / NL : (int)fdiv(iw, dN);
    const int e = iw - ch * N;
    if (kx0 + w < g.hx) spec[ch * cs + base_o + e * es_g + kx0 + w] = sm[((ch * Np + smap<NL>(e)) << lw) + w];
  }
}


// =========================== fused 2D column pass (float32, transposed scratch) =============
// The column (y) pass of the 2D apply on the transposed half spectrum spec[ch][kx][y]:
// every line (ch, kx) is contiguous.  A block takes KC columns (all 4 channels) with
// KC * N / 2 threads; KC is picked by the tile tuner (fewer columns per block give a
// single RVE more blocks, more give each block more work).
//   first DIF stage   global -> registers -> shared        (coalesced line loads)
//   middle DIF stages in shared memory
//   last DIF stage, projection (Eq. GFourier, Willot directions) and |xi|^2 multiply,
//   first DIT stage   three shared-memory phases (butterflies per line, then the projection
//                     per frequency position across the four channels, then butterflies)
//   middle DIT stages in shared memory
//   last DIT stage    shared -> registers -> global        (coalesced line stores)
// The radix of the last DIF / first DIT stage (span 1) is 8 for every compiled N.  Same
// arithmetic as k_col mode 1.
template <int N, int KC>
__global__ void __launch_bounds__(1024) k_col_fused2d(const __grid_constant__ ColGroup<float> grp) {
  const ColArgs<float> &a = grp.base;
  cpx<float> *const spec = grp.spec[blockIdx.y];
  const KrylovScalars *const ks = grp.ks[blockIdx.y];
  extern __shared__ unsigned char smraw[];
  cpx<float> *sm = reinterpret_cast<cpx<float> *>(smraw);
  if (ks && ks->done) return;
  constexpr StagePlan SP = stage_plan(N);
  constexpr int S = SP.S;
  static_assert(S >= 2 && SP.R[0] == 8 && SP.Ns[0] == 1, "fused column pass needs a radix-8 span-1 stage");
  static_assert(KC * N / 2 <= 1024, "at most 1024 threads (N / 2 per column)");
  constexpr int Np = N;  // smap slots
  constexpr int C = 4;             // channels: 3 strain (Mandel) + phase field
  constexpr int RT = SP.R[S - 1], NST = SP.Ns[S - 1];  // outermost stage: span N / RT
  constexpr int NBT = N / RT;
  const Geo &g = a.g;
  const int kx0 = blockIdx.x * KC;
  const int cs = g.hx * N;
  const cpx<float> *tw = (const cpx<float> *)a.plan.tw;
  // line (col, ch) of the block sits at (col * C + ch) * Np in shared memory

  // ---- first DIF stage: global -> registers -> shared --------------------------------------
  for (int b = threadIdx.x; b < KC * C * NBT; b += blockDim.x) {
    const int line = b / NBT, j = b - line * NBT;
    const int col = line / C, ch = line - col * C;
    const bool ok = kx0 + col < g.hx;
    const cpx<float> *src = spec + ch * cs + (kx0 + col) * N + j;
    cpx<float> v[RT];
#pragma unroll
    for (int r = 0; r < RT; ++r) v[r] = ok ? src[r * NST] : cpx<float>{0.f, 0.f};
    if constexpr (RT == 8) dft8(v, -1.f);
    else if constexpr (RT == 4) dft4(v, -1.f);
    else if constexpr (RT == 2) dft2(v);
    if (j != 0) {  // twiddle step N / (NST RT) = 1
      cpx<float> wt[RT];
      load_twiddles<float, RT>(tw, j, wt);
#pragma unroll
      for (int r = 1; r < RT; ++r) v[r] = cmul(v[r], wt[r]);
    }
    cpx<float> *dst = sm + line * Np;
#pragma unroll
    for (int r = 0; r < RT; ++r) dst[smap<N>(j + r * NST)] = v[r];
  }
  __syncthreads();
  ct_dif_range<float, N, S - 2, 1>(sm, KC * C, tw);

  // ---- middle: last DIF stage, projection, first DIT stage -------------------------------
  // Three shared-memory phases over N / 2 threads per column: (1) the span-1 radix-8 DIF
  // butterflies of every (column, channel) line; (2) at each frequency position, the projection
  // of the three strain channels (Willot directions) and the |xi|^2 multiply of the phase-field
  // channel; (3) the span-1 radix-8 DIT butterflies.  The same operations in the same order as
  // a thread holding all four channels of a butterfly, with a quarter of the registers.
  {
    const int t = threadIdx.x;
    for (int b = t; b < KC * C * (N / 8); b += blockDim.x) {
      const int line = b / (N / 8), q = b - line * (N / 8);
      cpx<float> *ln = sm + line * Np;
      cpx<float> v[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) v[r] = ln[smap<N>(8 * q + r)];
      dft8(v, -1.f);
#pragma unroll
      for (int r = 0; r < 8; ++r) ln[smap<N>(8 * q + r)] = v[r];
    }
    __syncthreads();
    for (int b = t; b < KC * N; b += blockDim.x) {
      const int col = b / N, pos = b - col * N;
      const int kx = kx0 + col;
      if (kx >= g.hx) continue;
      cpx<float> *base = sm + col * C * Np;
      const int sp = smap<N>(pos);
      {
        const float sc = (a.tab.xi2[0][kx] + a.tab.xi2[1][digit_rev_ct<N>(pos)]) * a.inv_n;
        const cpx<float> z = base[3 * Np + sp];
        base[3 * Np + sp] = {z.x * sc, z.y * sc};
      }
      int k[2] = {kx, digit_rev_ct<N>(pos)};
      float nv[3], xi2;
      willot_n<float, 2>(a.tab, k, nv, xi2);
      float re[3], im[3];
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const cpx<float> z = base[ch * Np + sp];
        re[ch] = z.x;
        im[ch] = z.y;
      }
      project_mandel<float, 3>(re, nv, a.inv_n);
      project_mandel<float, 3>(im, nv, a.inv_n);
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) base[ch * Np + sp] = {re[ch], im[ch]};
    }
    __syncthreads();
    for (int b = t; b < KC * C * (N / 8); b += blockDim.x) {
      const int line = b / (N / 8), q = b - line * (N / 8);
      cpx<float> *ln = sm + line * Np;
      cpx<float> v[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) v[r] = ln[smap<N>(8 * q + r)];
      dft8(v, 1.f);
#pragma unroll
      for (int r = 0; r < 8; ++r) ln[smap<N>(8 * q + r)] = v[r];
    }
  }
  __syncthreads();
  ct_dit_range<float, N, 1, S - 2>(sm, KC * C, tw);

  // ---- last DIT stage: shared -> registers -> global ---------------------------------------
  for (int b = threadIdx.x; b < KC * C * NBT; b += blockDim.x) {
    const int line = b / NBT, j = b - line * NBT;
    const int col = line / C, ch = line - col * C;
    const cpx<float> *src = sm + line * Np;
    cpx<float> v[RT];
#pragma unroll
    for (int r = 0; r < RT; ++r) v[r] = src[smap<N>(j + r * NST)];
    if (j != 0) {
      cpx<float> wt[RT];
      load_twiddles<float, RT>(tw, j, wt);
#pragma unroll
      for (int r = 1; r < RT; ++r) v[r] = cmul_conj(v[r], wt[r]);
    }
    if constexpr (RT == 8) dft8(v, 1.f);
    else if constexpr (RT == 4) dft4(v, 1.f);
    else if constexpr (RT == 2) dft2(v);
    if (kx0 + col < g.hx) {
      cpx<float> *dst = spec + ch * cs + (kx0 + col) * N + j;
#pragma unroll
      for (int r = 0; r < RT; ++r) dst[r * NST] = v[r];
    }
  }
}
