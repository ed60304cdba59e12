// Pointwise kernels of librve: the float64 constitutive update at a Newton iterate
// (Eqs. PlusNegPsi, gFunct, C_Calc, history, Delta_history), BiCGStab vector updates and
// scalar finalisation (Sec. 3.2), the Newton update of Algorithm 2, and reductions.
#include "rve_kern.cuh"
#include "krylov_fin.cuh"
#include "post.cuh"

namespace {
constexpr double kSqrt2 = 1.41421356237309504880;
constexpr double kInvSqrt2 = 0.70710678118654752440;

// Mandel <-> symmetric tensor (d x d, row-major e[i*3+j])
template <int M>
__device__ __forceinline__ void mandel_to_tensor(const double *mv, double *e) {
  if (M == 3) {
    e[0] = mv[0];
    e[1] = e[3] = mv[2] * kInvSqrt2;
    e[4] = mv[1];
  } else {
    e[0] = mv[0];
    e[4] = mv[1];
    e[8] = mv[2];
    e[5] = e[7] = mv[3] * kInvSqrt2;
    e[2] = e[6] = mv[4] * kInvSqrt2;
    e[1] = e[3] = mv[5] * kInvSqrt2;
  }
}
template <int M>
__device__ __forceinline__ void tensor_to_mandel(const double *e, double *mv) {
  if (M == 3) {
    mv[0] = e[0];
    mv[1] = e[4];
    mv[2] = e[1] * kSqrt2;
  } else {
    mv[0] = e[0];
    mv[1] = e[4];
    mv[2] = e[8];
    mv[3] = e[5] * kSqrt2;
    mv[4] = e[2] * kSqrt2;
    mv[5] = e[1] * kSqrt2;
  }
}

// Symmetric eigen-decomposition.  Q is row-major with eigenvectors as columns:
// e = Q diag(z) Q^T.  2D: closed form of the 2 x 2 block.  3D: cyclic Jacobi rotations.
__device__ __forceinline__ void eig2(const double *e, double *z, double *Q) {
  const double a = e[0], b = e[4], c = e[1];
  const double m = 0.5 * (a + b), h = 0.5 * (a - b);
  const double rad = sqrt(h * h + c * c);
  z[0] = m + rad;
  z[1] = m - rad;
  double ct = 1.0, st = 0.0;
  if (rad > 0.0) {
    const double c2 = h / rad, s2 = c / rad;  // cos 2t, sin 2t
    if (c2 >= 0.0) {
      ct = sqrt(0.5 * (1.0 + c2));
      st = s2 / (2.0 * ct);
    } else {
      st = sqrt(0.5 * (1.0 - c2));
      if (s2 < 0.0) st = -st;
      ct = s2 / (2.0 * st);
    }
  }
  // eigenvector of z0: (ct, st); of z1: (-st, ct)
  Q[0] = ct;
  Q[1] = -st;
  Q[3] = st;
  Q[4] = ct;
}

__device__ __forceinline__ void eig3(const double *e, double *z, double *Q) {
  double A[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) A[i] = e[i];
#pragma unroll
  for (int i = 0; i < 9; ++i) Q[i] = (i % 4 == 0) ? 1.0 : 0.0;
  double scale = fabs(A[0]) + fabs(A[4]) + fabs(A[8]) + fabs(A[1]) + fabs(A[2]) + fabs(A[5]);
  for (int sweep = 0; sweep < 12; ++sweep) {
    const double off = fabs(A[1]) + fabs(A[2]) + fabs(A[5]);
    if (off <= 1e-17 * scale || off == 0.0) break;
    const int P[3] = {0, 0, 1}, R[3] = {1, 2, 2};
    for (int k = 0; k < 3; ++k) {
      const int p = P[k], q = R[k];
      const double apq = A[p * 3 + q];
      if (apq == 0.0) continue;
      const double theta = (A[q * 3 + q] - A[p * 3 + p]) / (2.0 * apq);
      const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
      // A <- J^T A J with J the rotation in the (p, q) plane
      for (int r = 0; r < 3; ++r) {
        const double arp = A[r * 3 + p], arq = A[r * 3 + q];
        A[r * 3 + p] = c * arp - s * arq;
        A[r * 3 + q] = s * arp + c * arq;
      }
      for (int r = 0; r < 3; ++r) {
        const double apr = A[p * 3 + r], aqr = A[q * 3 + r];
        A[p * 3 + r] = c * apr - s * aqr;
        A[q * 3 + r] = s * apr + c * aqr;
      }
      for (int r = 0; r < 3; ++r) {
        const double qrp = Q[r * 3 + p], qrq = Q[r * 3 + q];
        Q[r * 3 + p] = c * qrp - s * qrq;
        Q[r * 3 + q] = s * qrp + c * qrq;
      }
    }
  }
  z[0] = A[0];
  z[1] = A[4];
  z[2] = A[8];
}

// divided difference of <x>+ (first-order Loewner matrix), tie rule H+((za+zb)/2); the
// differences in float64, the quotient in precision TT
template <typename TT>
__device__ __forceinline__ TT loewner_t(double za, double zb, double tie) {
  const double d = za - zb;
  if (fabs(d) <= tie) return (0.5 * (za + zb) > 0.0) ? (TT)1 : (TT)0;
  return (TT)(fmax(za, 0.0) - fmax(zb, 0.0)) / (TT)d;
}

}  // namespace

// =========================== constitutive update =============================================

// Per voxel: eps = eps_t + f E; spectral split; sigma = g sigma0+ + sigma0-; H = max(psi+, H^n);
// chi = [psi+ >= H^n]; tangent channels of the scaled Newton operator (TanIdx).
template <int M, typename TK>
__global__ void __launch_bounds__(256) k_constitutive(ConstArgs a, TK *tan) {
  using TI = TanIdx<M>;
  constexpr int D = (M == 3) ? 2 : 3;
  const long long n = a.g.n;
  double acc[M + 1];
#pragma unroll
  for (int k = 0; k <= M; ++k) acc[k] = 0;
  double mx[1] = {0.0};
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const uint8_t mb = a.mat[v];
    const bool notch = (mb & RVE_NOTCH_BIT) != 0;
    const int ph = mb & 0x7f;
    const double lam = a.ph.lam[ph], mu = a.ph.mu[ph], Gc = a.ph.Gc[ph];
    const double phi = a.phi[v], Hn = a.Hn[v];
    double em[M];
#pragma unroll
    for (int k = 0; k < M; ++k) em[k] = a.eps_t[k * n + v] + a.fM[k] * a.E;
    double e[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    mandel_to_tensor<M>(em, e);
    double z[3] = {0, 0, 0}, Q[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    // 2D: eigenvalues z0 >= z1 of the 2 x 2 block and the spectral projector onto z0's
    // eigenvector, P0 = (e - z1 I) / (z0 - z1) = I / 2 + (e - m I) / (2 rad), kept as
    // (P0_xx, P0_yy, P0_xy); the split needs no eigenvectors, the tangent builds them from P0
    // in the Krylov precision.  3D: cyclic Jacobi.
    double P0[3] = {1.0, 0.0, 0.0};
    if (D == 2) {
      const double mm = 0.5 * (e[0] + e[4]), hh = 0.5 * (e[0] - e[4]), cc = e[1];
      const double rad = sqrt(hh * hh + cc * cc);
      z[0] = mm + rad;
      z[1] = mm - rad;
      if (rad > 0.0) {
        const double ir = 0.5 / rad;
        P0[0] = 0.5 + hh * ir;
        P0[1] = 0.5 - hh * ir;
        P0[2] = cc * ir;
      }
    } else {
      eig3(e, z, Q);
    }
    const double tr = (D == 2) ? (e[0] + e[4]) : (e[0] + e[4] + e[8]);
    const double g = (1.0 - phi) * (1.0 - phi) + a.k_res;
    const double gp = -2.0 * (1.0 - phi);
    double psi_drive;
    double sig[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, sdrv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    double L[9];
    const double hp = tr > 0.0 ? 1.0 : 0.0;
    if (a.isotropic) {
      double ee = 0;
#pragma unroll
      for (int i = 0; i < 9; ++i) ee += e[i] * e[i];
      psi_drive = 0.5 * lam * tr * tr + mu * ee;
#pragma unroll
      for (int i = 0; i < 9; ++i) sdrv[i] = 2.0 * mu * e[i];
#pragma unroll
      for (int i = 0; i < D; ++i) sdrv[i * 4] += lam * tr;
#pragma unroll
      for (int i = 0; i < 9; ++i) sig[i] = g * sdrv[i];
    } else {
      double zp[3], zm[3];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        zp[i] = fmax(z[i], 0.0);
        zm[i] = fmin(z[i], 0.0);
      }
      const double trp = fmax(tr, 0.0), trm = fmin(tr, 0.0);
      psi_drive = 0.5 * lam * trp * trp;
#pragma unroll
      for (int i = 0; i < D; ++i) psi_drive += mu * zp[i] * zp[i];
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
          double ep = 0, emn = 0;
          if (D == 2) {  // e+- = <z0>+- P0 + <z1>+- (I - P0)
            const double p = i == j ? P0[i] : P0[2];
            const double q = (i == j ? 1.0 : 0.0) - p;
            ep = zp[0] * p + zp[1] * q;
            emn = zm[0] * p + zm[1] * q;
          } else {
#pragma unroll
            for (int k = 0; k < D; ++k) {
              ep += Q[i * 3 + k] * zp[k] * Q[j * 3 + k];
              emn += Q[i * 3 + k] * zm[k] * Q[j * 3 + k];
            }
          }
          sdrv[i * 3 + j] = 2.0 * mu * ep + (i == j ? lam * trp : 0.0);
          sig[i * 3 + j] = g * sdrv[i * 3 + j] + 2.0 * mu * emn + (i == j ? lam * trm : 0.0);
        }
      double zmax = 0;
#pragma unroll
      for (int i = 0; i < D; ++i) zmax = fmax(zmax, fabs(z[i]));
      const double tie = 1e-12 * zmax;
      // L only enters the tangent: the tie test and both differences in float64, the
      // quotient in the Krylov precision (one float64 division fewer per pair in MIXED)
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) L[i * 3 + j] = (double)loewner_t<TK>(z[i], z[j], tie);
    }
    const double H = fmax(psi_drive, Hn);
    const double chi = (psi_drive >= Hn) ? 1.0 : 0.0;
    double sm[M], dm[M];
    tensor_to_mandel<M>(sig, sm);
    tensor_to_mandel<M>(sdrv, dm);
#pragma unroll
    for (int k = 0; k < M; ++k) {
      a.sigma[k * n + v] = sm[k];
      acc[k] += sm[k];
      acc[M] += (a.s1 * sm[k]) * (a.s1 * sm[k]);
    }
    a.H[v] = H;
    if (!notch) mx[0] = fmax(mx[0], 2.0 * psi_drive / (Gc / a.ell));
    // tangent in Mandel form: column kb = C_t applied to the kb-th Mandel basis tensor,
    // evaluated in the Krylov precision TK (it only enters the Newton operator)
    TK Ct[M][M];
    {
      using TT = TK;
      const TT gT = (TT)g, muT = (TT)mu, lamT = (TT)lam;
      TT Qt[9], Lt[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        Qt[i] = (TT)Q[i];
        Lt[i] = a.isotropic ? (TT)0 : (TT)L[i];
      }
      if (D == 2 && !a.isotropic) {
        // eigenvectors (ct, st) of z0 and (-st, ct) of z1 from P0: ct^2 = P0_xx,
        // st^2 = P0_yy, ct st = P0_xy, taking the root of the larger diagonal entry
        const TT p00 = (TT)P0[0], p11 = (TT)P0[1], p01 = (TT)P0[2];
        TT ct, st;
        if (p00 >= p11) {
          ct = sqrt(p00);
          st = p01 / ct;
        } else {
          st = sqrt(p11);
          if (p01 < (TT)0) st = -st;
          ct = p01 / st;
        }
        Qt[0] = ct;
        Qt[1] = -st;
        Qt[3] = st;
        Qt[4] = ct;
      }
      const TT volc = a.isotropic ? gT * lamT : (TT)(g * lam * hp + lam * (1.0 - hp));
#pragma unroll
      for (int kb = 0; kb < M; ++kb) {
        // basis tensor: unit on (i0, i0) for kb < D, else (e_i0 e_j0 + e_j0 e_i0) / sqrt 2
        int i0, j0;
        if (kb < D) {
          i0 = j0 = kb;
        } else if (M == 3) {
          i0 = 0;
          j0 = 1;
        } else {
          i0 = kb == 3 ? 1 : 0;
          j0 = kb == 5 ? 1 : 2;
        }
        const TT w = kb < D ? (TT)1 : (TT)kInvSqrt2;
        const TT trd = kb < D ? (TT)1 : (TT)0;
        TT res[3][3];
        if (a.isotropic) {
#pragma unroll
          for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
              const TT dij = ((i == i0 && j == j0) || (i == j0 && j == i0)) ? w : (TT)0;
              res[i][j] = (TT)2 * gT * muT * dij + (i == j ? volc * trd : (TT)0);
            }
        } else {
          // Dp = Q (L o (Q^T d Q)) Q^T with (Q^T d Q)_pq = w (Q_i0p Q_j0q + Q_j0p Q_i0q) (halved on the diagonal)
          TT Mt[3][3];
#pragma unroll
          for (int p = 0; p < D; ++p)
#pragma unroll
            for (int q = 0; q < D; ++q) {
              TT A = Qt[i0 * 3 + p] * Qt[j0 * 3 + q];
              if (kb >= D) A += Qt[j0 * 3 + p] * Qt[i0 * 3 + q];
              Mt[p][q] = w * A * Lt[p * 3 + q];
            }
#pragma unroll
          for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
              TT dp = 0;
#pragma unroll
              for (int p = 0; p < D; ++p)
#pragma unroll
                for (int q = 0; q < D; ++q) dp += Qt[i * 3 + p] * Mt[p][q] * Qt[j * 3 + q];
              const TT dij = ((i == i0 && j == j0) || (i == j0 && j == i0)) ? w : (TT)0;
              res[i][j] = (TT)2 * gT * muT * dp + (TT)2 * muT * (dij - dp) + (i == j ? volc * trd : (TT)0);
            }
        }
        // Mandel column
        Ct[0][kb] = res[0][0];
        Ct[1][kb] = res[1][1];
        if (M == 3) {
          Ct[2][kb] = res[0][1] * (TT)kSqrt2;
        } else {
          Ct[2][kb] = res[2][2];
          Ct[3][kb] = res[1][2] * (TT)kSqrt2;
          Ct[4][kb] = res[0][2] * (TT)kSqrt2;
          Ct[5][kb] = res[0][1] * (TT)kSqrt2;
        }
      }
    }
    int idx = 0;
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
      for (int j = i; j < M; ++j) {
        tan[idx * n + v] = (TK)a.s1 * (TK)0.5 * (Ct[i][j] + Ct[j][i]);
        ++idx;
      }
    // row scaling of the phase-field row for the tangent channels, evaluated in the Krylov
    // precision (float64 sums, one TK division)
    const TK s2 = notch ? (TK)1 : (TK)1 / (TK)(Gc / a.ell + 2.0 * H + Gc * a.ell * a.Lbar);
#pragma unroll
    for (int k = 0; k < M; ++k) tan[(TI::SF + k) * n + v] = (TK)(notch ? 0.0 : a.s1 * gp * dm[k]);
    tan[TI::KAPPA * n + v] = notch ? (TK)0 : (TK)chi * s2 / (TK)a.s1;
    tan[TI::A * n + v] = notch ? (TK)0 : s2 * (TK)(Gc / a.ell + 2.0 * H);
    tan[TI::B * n + v] = notch ? (TK)0 : s2 * (TK)Gc * (TK)a.ell;
    tan[TI::NOTCH * n + v] = (TK)(notch ? 1.0 : 0.0);
  }
  block_partials<M + 1>(acc, a.part, gridDim.x, blockIdx.x);
  block_max_partials<1>(mx, a.part_max, gridDim.x, blockIdx.x);
}

// =========================== reductions ======================================================
// Deterministic fixed-order sum of G partials (one block, any G), krylov_fin.cuh.
__device__ double sum_partials(const double *p, int G) { return sum_partials_t<false>(p, G); }
__device__ double max_partials(const double *p, int G) {
  __shared__ double red[256];
  double s = -1e308;
  for (int i = threadIdx.x; i < G; i += blockDim.x) s = fmax(s, p[i]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// out[q] = sum (or max if is_max) of part[q * G .. q * G + G), q < NQ.  <<<1, 256>>>
__global__ void k_reduce(const double *part, int G, int NQ, int is_max, double *out) {
  for (int q = 0; q < NQ; ++q) {
    const double r = is_max ? max_partials(part + (size_t)q * G, G) : sum_partials(part + (size_t)q * G, G);
    if (threadIdx.x == 0) out[q] = r;
  }
}

__global__ void k_reduce_list(ReduceList L, double *out) {
  for (int i = 0; i < L.n; ++i) {
    const ReduceSeg &sg = L.s[i];
    for (int q = 0; q < sg.NQ; ++q) {
      const double *p = sg.part + (size_t)q * sg.G;
      const double r = sg.is_max ? max_partials(p, sg.G) : sum_partials(p, sg.G);
      if (threadIdx.x == 0) out[sg.off + q] = r;
    }
  }
}

// =========================== BiCGStab ========================================================
// Vector of the Krylov space: c channels of n values (type TK) + an E slot in KrylovScalars.

// SplitMix64 (Steele, Lea, Flood 2014): shadow direction zeta in [-1, 1)
__device__ __forceinline__ double unit_hash(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * 0x1.0p-52 - 1.0;
}

// (Re)start of BiCGStab: rhat = r + sqrt(|r|^2 / N) zeta_seed (ks->rn2 = |r|^2 set before),
// p = v = 0, x = 0 unless restarting from a kept iterate; partial (rhat, r).
// zeta_seed of component i is unit_hash(i + seed * N), N = c n + 1 (E slot: i = c n).
template <typename TK>
__global__ void k_kinit(KvArgs<TK> a, int seed, int zero_x) {
  const double Ntot = (double)a.len + 1.0;
  const double cz = sqrt(a.ks->rn2 / Ntot);
  const unsigned long long off = (unsigned long long)seed * (unsigned long long)(a.len + 1);
  double acc[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.len;
       i += (long long)gridDim.x * blockDim.x) {
    const TK r = a.r[i];
    const TK rh = (TK)((double)r + cz * unit_hash((unsigned long long)i + off));
    a.rhat[i] = rh;
    if (zero_x) a.x[i] = 0;
    a.p[i] = 0;
    a.v[i] = 0;
    acc[0] += (double)rh * (double)r;
  }
  block_partials<1>(acc, a.part, gridDim.x, blockIdx.x);
}

// <<<1,256>>>: rhat_E, rho = (rhat, r), beta = rho, pE = rE (first iteration after a
// (re)start: p = v = 0, alpha = omega = 1).  len = c * n.
__global__ void k_kfin_init(KrylovScalars *ks, const double *part, int G, long long len, int seed,
                            int zero_x) {
  const double d = sum_partials(part, G);
  if (threadIdx.x == 0) {
    const double cz = sqrt(ks->rn2 / ((double)len + 1.0));
    const unsigned long long off = (unsigned long long)seed * (unsigned long long)(len + 1);
    ks->rhE = ks->rE + cz * unit_hash((unsigned long long)len + off);
    const double rho = ks->fault_rho0 ? 0.0 : d + ks->rhE * ks->rE;
    ks->rho = rho;
    ks->beta = rho;
    ks->alpha = 1.0;
    ks->omega = 1.0;
    if (zero_x) ks->xE = 0.0;
    ks->pE = ks->rE;
    ks->vE = 0.0;
    ks->status = 0;
    ks->done = 0;
    ks->pending = 0;
    if (ks->rn2 == 0.0) {
      ks->done = 1;
    } else if (rho == 0.0) {
      ks->done = 1;
      ks->status = 2;
    }
  }
}

// restart: r = b - t (t = A x just computed), partial |r|^2
template <typename TK>
__global__ void k_kresid(long long len, const TK *b, const TK *t, TK *r, double *part) {
  double acc[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    const TK v = b[i] - t[i];
    r[i] = v;
    acc[0] += (double)v * (double)v;
  }
  block_partials<1>(acc, part, gridDim.x, blockIdx.x);
}

// |t|^2 + (A x)_E^2 of an apply with x = (0, 0, 1): column norm of the E unknown
template <typename TK>
__global__ void k_norm2(long long len, const TK *t, double *part) {
  double acc[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = (double)t[i];
    acc[0] += v * v;
  }
  block_partials<1>(acc, part, gridDim.x, blockIdx.x);
}

// partial max |t_i| (step bound on the phase-field channel of a Newton step)
template <typename TK>
__global__ void k_maxabs(long long len, const TK *t, double *part) {
  double acc[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    acc[0] = fmax(acc[0], fabs((double)t[i]));
  block_max_partials<1>(acc, part, gridDim.x, blockIdx.x);
}

// restart: rE = bE - (A x)_E, rn2 = |r|^2
__global__ void k_kfin_resid(KrylovScalars *ks, const double *part_app, int Gx, const double *part_kv,
                             int Gpw) {
  const double wdp = sum_partials(part_app, Gx);
  const double rr = sum_partials(part_kv, Gpw);
  if (threadIdx.x == 0) {
    const double yE = ks->strain ? ks->xE : ks->s3 * wdp;  // strain control: no E scaling
    ks->rE = ks->bE - yE;
    ks->rn2 = rr + ks->rE * ks->rE;
  }
}

// x += alpha p + omega s; r = s - omega t; partials |r|^2, (rhat, r)
template <typename TK>
__global__ void k_kxr(const __grid_constant__ KvGroup<TK> grp) {
  const KvArgs<TK> &a = grp.m[blockIdx.y];
  if (a.ks->done) return;
  const TK al = (TK)a.ks->alpha, om = (TK)a.ks->omega;
  TK rr = 0, rhr = 0;  // per-thread and warp sums in TK, block and grid sums in float64
  long long i0 = 0;
  if constexpr (sizeof(TK) == 4) {
    // 16-byte accesses over the bulk when every vector is 16-byte aligned
    const unsigned long long al16 = (unsigned long long)a.x | (unsigned long long)a.p | (unsigned long long)a.s |
                                    (unsigned long long)a.t | (unsigned long long)a.r | (unsigned long long)a.rhat;
    if ((al16 & 15) == 0) {
      const long long n4 = a.len / 4;
      float4 *x4 = reinterpret_cast<float4 *>(a.x), *r4 = reinterpret_cast<float4 *>(a.r);
      const float4 *p4 = reinterpret_cast<const float4 *>(a.p), *s4 = reinterpret_cast<const float4 *>(a.s);
      const float4 *t4 = reinterpret_cast<const float4 *>(a.t), *h4 = reinterpret_cast<const float4 *>(a.rhat);
      for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
           i += (long long)gridDim.x * blockDim.x) {
        const float4 sv = s4[i], pv = p4[i], tv = t4[i], hv = h4[i];
        float4 xv = x4[i];
        xv.x += al * pv.x + om * sv.x;
        xv.y += al * pv.y + om * sv.y;
        xv.z += al * pv.z + om * sv.z;
        xv.w += al * pv.w + om * sv.w;
        x4[i] = xv;
        const float4 rv = make_float4(sv.x - om * tv.x, sv.y - om * tv.y, sv.z - om * tv.z, sv.w - om * tv.w);
        r4[i] = rv;
        rr += rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w;
        rhr += hv.x * rv.x + hv.y * rv.y + hv.z * rv.z + hv.w * rv.w;
      }
      i0 = 4 * n4;
    }
  }
  for (long long i = i0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.len;
       i += (long long)gridDim.x * blockDim.x) {
    const TK s = a.s[i];
    a.x[i] += al * a.p[i] + om * s;
    const TK r = s - om * a.t[i];
    a.r[i] = r;
    rr += r * r;
    rhr += a.rhat[i] * r;
  }
  const TK acc[2] = {rr, rhr};
  block_partials_k<TK, 2>(acc, a.part, gridDim.x, blockIdx.x);
  // the member's last block to finish runs the convergence test (no separate finaliser)
  if (a.arrive && last_block_arrives(a.arrive, gridDim.x)) fin_conv<true>(a.ks, a.part, gridDim.x);
}

// Close of a float32 chunk: the vector update the last iteration left pending,
// x += alpha p + omega s, r = s - omega t (also after the solve has stopped: done is not
// checked); the member's last block clears the flag.
template <typename TK>
__global__ void k_kx_finish(const __grid_constant__ KvGroup<TK> grp) {
  const KvArgs<TK> &a = grp.m[blockIdx.y];
  if (!a.ks->pending) return;
  const TK al = (TK)a.ks->alpha, om = (TK)a.ks->omega;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.len;
       i += (long long)gridDim.x * blockDim.x) {
    const TK s = a.s[i];
    a.x[i] += al * a.p[i] + om * s;
    a.r[i] = s - om * a.t[i];
  }
  if (last_block_arrives(a.arrive, gridDim.x) && threadIdx.x == 0) a.ks->pending = 0;
}

// =========================== Newton update ===================================================
// q_trial += a dq with dq the Krylov solution; partials |dq_eps|^2, |dq_phi|^2,
// |eps_new|^2 (total strain eps_tilde + f E_new, Mandel norm), |phi_new|^2
template <typename TK>
__global__ void k_newton_update(long long n, int m, const TK *xe, const TK *xp, double step, double *eps_t,
                                double *phi, const double *fM, double E_new, double *part) {
  // xe: m strain channels of the step (stride n), xp: its phase-field channel
  double acc[4] = {0, 0, 0, 0};
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    for (int k = 0; k < m; ++k) {
      const double d = (double)xe[k * n + v];
      const double e = eps_t[k * n + v] + step * d;
      eps_t[k * n + v] = e;
      const double et = e + fM[k] * E_new;
      acc[0] += d * d;
      acc[2] += et * et;
    }
    const double dp = (double)xp[v];
    const double p = phi[v] + step * dp;
    phi[v] = p;
    acc[1] += dp * dp;
    acc[3] += p * p;
  }
  block_partials<4>(acc, part, gridDim.x, blockIdx.x);
}

// Staggered sub-solves (Algorithm 1) on the monolithic operator: after a linearisation,
// mode 1 (mechanics at fixed phi) turns every phase-field row into an identity row with a
// zero right-hand side; mode 2 (phase field at fixed H) drops the strain rows (zero tangent,
// zero right-hand side) and the strain coupling of the phase-field rows.
template <int M, typename TK>
__global__ void k_stag_mask(long long n, int mode, TK *tan, TK *rhs) {
  using TI = TanIdx<M>;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    if (mode == 1) {
      tan[TI::NOTCH * n + v] = (TK)1;
      tan[TI::KAPPA * n + v] = (TK)0;
      tan[TI::A * n + v] = (TK)0;
      tan[TI::W * n + v] = (TK)0;
      tan[TI::B * n + v] = (TK)0;
#pragma unroll
      for (int k = 0; k < M; ++k) tan[(TI::SF + k) * n + v] = (TK)0;
      rhs[M * n + v] = (TK)0;
    } else {
#pragma unroll
      for (int k = 0; k < TI::NC; ++k) tan[k * n + v] = (TK)0;
#pragma unroll
      for (int k = 0; k < M; ++k) {
        tan[(TI::SF + k) * n + v] = (TK)0;
        rhs[k * n + v] = (TK)0;
      }
      tan[TI::KAPPA * n + v] = (TK)0;
    }
  }
}

// =========================== small helpers ===================================================
template <typename TA, typename TB>
__global__ void k_convert(long long len, const TA *a, TB *b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (TB)a[i];
}

// total strain eps = eps_tilde + f E (m channels)
__global__ void k_total_strain(long long n, int m, const double *eps_t, const double *fM, double E,
                               double *out) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x)
    for (int k = 0; k < m; ++k) out[k * n + v] = eps_t[k * n + v] + fM[k] * E;
}

// =========================== J-integral (2D post-process) =====================================
// Rotation spectrum: the compatibility relations d1 w = d1 e12 - d2 e11, d2 w = d1 e22 - d2 e12
// give w-hat = [xi1 (xi1 e12 - xi2 e11) + xi2 (xi1 e22 - xi2 e12)] / |xi|^2 with the standard
// frequencies xi = 2 pi k / N (Nyquist component 0); w-hat = 0 at |xi| = 0.
__global__ void k_rot_spec(RotArgs a) {
  const Geo &g = a.g;
  const long long tot = (long long)g.ny * g.hx;
  const long long cs = (long long)g.rows * g.hx;
  const double two_pi = 6.283185307179586476925;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(i / g.hx), kx = (int)(i - (long long)p * g.hx);
    const int ky = a.yrev[p];
    const double x1 = (2 * kx == g.nx) ? 0.0 : two_pi * (double)kx / (double)g.nx;
    const int ks = (2 * ky < g.ny) ? ky : ky - g.ny;
    const double x2 = (2 * ky == g.ny) ? 0.0 : two_pi * (double)ks / (double)g.ny;
    const double q = x1 * x1 + x2 * x2;
    const cpx<double> e11 = a.spec[i], e22 = a.spec[cs + i], m12 = a.spec[2 * cs + i];
    const double e12r = m12.x * kInvSqrt2, e12i = m12.y * kInvSqrt2;
    cpx<double> w = {0.0, 0.0};
    if (q > 0.0) {
      const double s = a.inv_n / q;
      w.x = (x1 * (x1 * e12r - x2 * e11.x) + x2 * (x1 * e22.x - x2 * e12r)) * s;
      w.y = (x1 * (x1 * e12i - x2 * e11.y) + x2 * (x1 * e22.y - x2 * e12i)) * s;
    }
    a.spec[i] = w;
  }
}

// Contour sum of (W n1 - t . d1 u) over the rectangle's sides (right, top, left, bottom; each
// side from its first to its last voxel, the two end voxels weighted 1/2), with W = g psi0+ +
// psi0- (spectral split) or g psi0 (isotropic), sigma the degraded stress, and
// d1 u1 = E f11 + e~11, d1 u2 = E f21 + e~12 + w.  One block of 256 threads; the per-thread
// sums are added in a fixed order.
__global__ void __launch_bounds__(256) k_j_contour(JArgs a) {
  __shared__ double red[256];
  const int nxs = a.x1 - a.x0 + 1, nys = a.y1 - a.y0 + 1;
  const int tot = 2 * nxs + 2 * nys;
  const long long n = a.g.n;
  double acc = 0.0;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    int side, t, len;
    if (i < nys) { side = 0; t = i; len = nys; }
    else if (i < nys + nxs) { side = 1; t = i - nys; len = nxs; }
    else if (i < 2 * nys + nxs) { side = 2; t = i - nys - nxs; len = nys; }
    else { side = 3; t = i - 2 * nys - nxs; len = nxs; }
    int x, y;
    double n1 = 0.0, n2 = 0.0;
    switch (side) {
      case 0: x = a.x1; y = a.y0 + t; n1 = 1.0; break;
      case 1: x = a.x0 + t; y = a.y1; n2 = 1.0; break;
      case 2: x = a.x0; y = a.y0 + t; n1 = -1.0; break;
      default: x = a.x0 + t; y = a.y0; n2 = -1.0; break;
    }
    const double wgt = (t == 0 || t == len - 1) ? 0.5 : 1.0;
    const long long v = (long long)y * a.g.nx + x;
    const int ph = a.mat[v] & 0x7f;
    const double lam = a.ph.lam[ph], mu = a.ph.mu[ph];
    const double phi = a.phi[v];
    const double gd = (1.0 - phi) * (1.0 - phi) + a.k_res;
    double em[3], e[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 3; ++k) em[k] = a.eps_t[k * n + v] + a.fM[k] * a.E;
    mandel_to_tensor<3>(em, e);
    const double tr = e[0] + e[4];
    double s11, s22, s12, W;
    if (a.isotropic) {
      W = gd * (0.5 * lam * tr * tr + mu * (e[0] * e[0] + e[4] * e[4] + 2.0 * e[1] * e[1]));
      s11 = gd * (2.0 * mu * e[0] + lam * tr);
      s22 = gd * (2.0 * mu * e[4] + lam * tr);
      s12 = gd * 2.0 * mu * e[1];
    } else {
      double z[3] = {0, 0, 0}, Q[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
      eig2(e, z, Q);
      const double trp = fmax(tr, 0.0), trm = fmin(tr, 0.0);
      double sp[3] = {lam * trp, lam * trp, 0.0}, sn[3] = {lam * trm, lam * trm, 0.0};  // 11, 22, 12
      double psip = 0.5 * lam * trp * trp, psim = 0.5 * lam * trm * trm;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const double zp = fmax(z[k], 0.0), zm = fmin(z[k], 0.0);
        const double q1 = Q[k], q2 = Q[3 + k];  // eigenvector k (column k of Q)
        psip += mu * zp * zp;
        psim += mu * zm * zm;
        sp[0] += 2.0 * mu * zp * q1 * q1;
        sp[1] += 2.0 * mu * zp * q2 * q2;
        sp[2] += 2.0 * mu * zp * q1 * q2;
        sn[0] += 2.0 * mu * zm * q1 * q1;
        sn[1] += 2.0 * mu * zm * q2 * q2;
        sn[2] += 2.0 * mu * zm * q1 * q2;
      }
      W = gd * psip + psim;
      s11 = gd * sp[0] + sn[0];
      s22 = gd * sp[1] + sn[1];
      s12 = gd * sp[2] + sn[2];
    }
    const double du1 = a.E * a.fM[0] + a.eps_t[v];
    const double du2 = (a.E * a.fM[2] + a.eps_t[2 * n + v]) * kInvSqrt2 + a.w[v];
    const double t1 = s11 * n1 + s12 * n2, t2 = s12 * n1 + s22 * n2;
    acc += wgt * (W * n1 - (t1 * du1 + t2 * du2));
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *a.out = red[0];
}

// =========================== energy-controlled constraint (Eq. SystemDisc) =====================
// Spectral derivative D_a of Eq. newGammaFourier: multiplier s_a = i xi_a (xi = 2 pi k / N),
// except the real |xi_a| = pi at the Nyquist index of an even axis (keeps the field real and
// Parseval exact).  The adjoint multiplies by conj(s_a).
__device__ __forceinline__ void deriv_symbol(int k, int N, double &re, double &im) {
  const double two_pi = 6.283185307179586476925;
  if (2 * k == N) {
    re = 0.5 * two_pi;
    im = 0.0;
    return;
  }
  const int ks = (2 * k < N) ? k : k - N;
  re = 0.0;
  im = two_pi * (double)ks / (double)N;
}

template <int M>
__device__ __forceinline__ void spec_freqs(const SpecOpArgs &a, long long i, int *k) {
  const Geo &g = a.g;
  const int kx = (int)(i % g.hx);
  const long long r = i / g.hx;
  k[0] = kx;
  if (M == 3) {
    k[1] = a.yrev[r];
  } else {
    k[1] = a.yrev[(int)(r % g.ny)];
    k[2] = a.zrev[(int)(r / g.ny)];
  }
}

// channels a < d <- s_a * (channel m = phi-hat) / n
template <int M>
__global__ void k_grad_spec(SpecOpArgs a) {
  constexpr int D = (M == 3) ? 2 : 3;
  const Geo &g = a.g;
  const long long cs = (long long)g.rows * g.hx;
  const int Ns[3] = {g.nx, g.ny, g.nz};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cs;
       i += (long long)gridDim.x * blockDim.x) {
    int k[3];
    spec_freqs<M>(a, i, k);
    const cpx<double> p = a.spec[M * cs + i];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      double sr, si;
      deriv_symbol(k[d], Ns[d], sr, si);
      a.spec[d * cs + i] = {(sr * p.x - si * p.y) * a.inv_n, (sr * p.y + si * p.x) * a.inv_n};
    }
  }
}

// channel 0 <- sum_a conj(s_a) * channel a / n
template <int M>
__global__ void k_div_spec(SpecOpArgs a) {
  constexpr int D = (M == 3) ? 2 : 3;
  const Geo &g = a.g;
  const long long cs = (long long)g.rows * g.hx;
  const int Ns[3] = {g.nx, g.ny, g.nz};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cs;
       i += (long long)gridDim.x * blockDim.x) {
    int k[3];
    spec_freqs<M>(a, i, k);
    double re = 0.0, im = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      double sr, si;
      deriv_symbol(k[d], Ns[d], sr, si);
      const cpx<double> q = a.spec[d * cs + i];
      re += sr * q.x + si * q.y;
      im += sr * q.y - si * q.x;
    }
    a.spec[i] = {re * a.inv_n, im * a.inv_n};
  }
}

// buf[a] = D_a phi -> G_c D_a phi; partial 0: sum G_c (phi^2 / (2 l) + (l / 2) |D phi|^2)
template <int M>
__global__ void __launch_bounds__(256) k_energy_flux(EnergyArgs a) {
  constexpr int D = (M == 3) ? 2 : 3;
  const long long n = a.g.n;
  double acc[1] = {0.0};
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const double Gc = a.ph.Gc[a.mat[v] & 0x7f];
    const double p = a.phi[v];
    double g2 = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const double t = a.buf[d * n + v];
      g2 += t * t;
      a.buf[d * n + v] = Gc * t;
    }
    acc[0] += Gc * (p * p / (2.0 * a.ell) + 0.5 * a.ell * g2);
  }
  block_partials<1>(acc, a.part, gridDim.x, blockIdx.x);
}

// buf[0] = sum_a D_a^T (G_c D_a phi):  w = G_c phi / l + l buf[0] (0 on the notch) into the
// constraint-row channel of the tangent; partial 1: |w|^2
template <int M, typename TK>
__global__ void __launch_bounds__(256) k_energy_w(EnergyArgs a, TK *tan) {
  using TI = TanIdx<M>;
  const long long n = a.g.n;
  double acc[1] = {0.0};
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const uint8_t mb = a.mat[v];
    const bool notch = (mb & RVE_NOTCH_BIT) != 0;
    const double Gc = a.ph.Gc[mb & 0x7f];
    const double w = notch ? 0.0 : Gc * a.phi[v] / a.ell + a.ell * a.buf[v];
    tan[TI::W * n + v] = (TK)w;
    acc[0] += w * w;
  }
  block_partials<1>(acc, a.part + gridDim.x, gridDim.x, blockIdx.x);
}

template __global__ void k_grad_spec<3>(SpecOpArgs);
template __global__ void k_grad_spec<6>(SpecOpArgs);
template __global__ void k_div_spec<3>(SpecOpArgs);
template __global__ void k_div_spec<6>(SpecOpArgs);
template __global__ void k_energy_flux<3>(EnergyArgs);
template __global__ void k_energy_flux<6>(EnergyArgs);
template __global__ void k_energy_w<3, float>(EnergyArgs, float *);
template __global__ void k_energy_w<6, float>(EnergyArgs, float *);
template __global__ void k_energy_w<3, double>(EnergyArgs, double *);
template __global__ void k_energy_w<6, double>(EnergyArgs, double *);

template __global__ void k_constitutive<3, float>(ConstArgs, float *);
template __global__ void k_constitutive<6, float>(ConstArgs, float *);
template __global__ void k_constitutive<3, double>(ConstArgs, double *);
template __global__ void k_constitutive<6, double>(ConstArgs, double *);
template __global__ void k_kinit<float>(KvArgs<float>, int, int);
template __global__ void k_kinit<double>(KvArgs<double>, int, int);
template __global__ void k_maxabs<float>(long long, const float *, double *);
template __global__ void k_maxabs<double>(long long, const double *, double *);
template __global__ void k_norm2<float>(long long, const float *, double *);
template __global__ void k_norm2<double>(long long, const double *, double *);
template __global__ void k_kresid<float>(long long, const float *, const float *, float *, double *);
template __global__ void k_kresid<double>(long long, const double *, const double *, double *, double *);
template __global__ void k_kxr<float>(const __grid_constant__ KvGroup<float>);
template __global__ void k_kx_finish<float>(const __grid_constant__ KvGroup<float>);
template __global__ void k_kx_finish<double>(const __grid_constant__ KvGroup<double>);
template __global__ void k_kxr<double>(const __grid_constant__ KvGroup<double>);
template __global__ void k_newton_update<float>(long long, int, const float *, const float *, double,
                                                double *, double *, const double *, double, double *);
template __global__ void k_newton_update<double>(long long, int, const double *, const double *, double,
                                                 double *, double *, const double *, double, double *);
template __global__ void k_convert<double, float>(long long, const double *, float *);
template __global__ void k_convert<float, double>(long long, const float *, double *);
template __global__ void k_convert<double, double>(long long, const double *, double *);
template __global__ void k_stag_mask<3, float>(long long, int, float *, float *);
template __global__ void k_stag_mask<6, float>(long long, int, float *, float *);
template __global__ void k_stag_mask<3, double>(long long, int, double *, double *);
template __global__ void k_stag_mask<6, double>(long long, int, double *, double *);
