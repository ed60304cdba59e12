// BiCGStab finalisation (Sec. 3.2): the deterministic sum of per-block partials and the
// scalar updates that follow each apply of an iteration and its vector update.  The same
// device functions serve the single-block finaliser kernels (kernels_pw.cu) and the last
// block of the kernel that produced the partials (fft_passes.cuh, k_kxr), which finalises
// in place of a separate launch.
#pragma once
#include "rve_kern.cuh"

// Deterministic fixed-order sum of G partials (one block of 256 threads, any G): Neumaier-
// compensated per-thread sums, then a tree that carries (sum, compensation) pairs and merges
// two sums with Knuth's TwoSum (exact rounding error of a + b), so the compensation of every
// partial reaches the result.  CG: the partials were written by other blocks of the running
// kernel, so they are read past L1 (ld.global.cg).
template <bool CG>
__device__ __forceinline__ double sum_partials_t(const double *p, int G) {
  __shared__ double red[256], cmp[256];
  double s = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < G; i += blockDim.x) {
    const double x = CG ? __ldcg(p + i) : p[i];
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
  red[threadIdx.x] = s;
  cmp[threadIdx.x] = c;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double a = red[threadIdx.x], b = red[threadIdx.x + o];
      const double t = a + b;
      const double bv = t - a;
      const double err = (a - (t - bv)) + (b - bv);
      red[threadIdx.x] = t;
      cmp[threadIdx.x] += cmp[threadIdx.x + o] + err;
    }
    __syncthreads();
  }
  const double r = red[0] + cmp[0];
  __syncthreads();
  return r;
}

// Last-block detection over the blocks of one group member (nblocks of them): every block
// publishes its partials (the caller wrote them), fences, and counts itself in; the block that
// brings the count to nblocks returns true (uniformly for its threads) and resets the counter
// for the next launch.  The counter starts at 0 (zeroed when the handle is created).
__device__ __forceinline__ bool last_block_arrives(unsigned int *ctr, unsigned int nblocks) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int prev = atomicAdd(ctr, 1u);
    last = prev == nblocks - 1 ? 1 : 0;
    if (last) *ctr = 0u;
  }
  __syncthreads();
  return last != 0;
}

// after apply(p -> v): vE = s3 sum(w dphi), alpha = rho / (rhat, v), sE = rE - alpha vE.
// part: G partials of sum w dphi, then G of (rhat, v).
template <bool CG>
__device__ __forceinline__ void fin_alpha(KrylovScalars *ks, const double *part, int G) {
  const double wdp = sum_partials_t<CG>(part, G);
  const double rv = sum_partials_t<CG>(part + G, G);
  if (threadIdx.x == 0) {
    ks->vE = ks->strain ? ks->pE : ks->s3 * wdp;
    const double rvt = rv + ks->rhE * ks->vE;
    if (rvt == 0.0) {
      ks->done = 1;
      ks->status = 2;
      return;
    }
    ks->alpha = ks->rho / rvt;
    ks->sE = ks->rE - ks->alpha * ks->vE;
  }
}

// alpha update of a float32 chunk iteration: as fin_alpha, and the pending vector update of
// the previous iteration, which the x-forward pass just applied, is cleared.
template <bool CG>
__device__ __forceinline__ void fin_alpha_clear(KrylovScalars *ks, const double *part, int G) {
  fin_alpha<CG>(ks, part, G);
  if (threadIdx.x == 0) ks->pending = 0;
}

// after apply(s -> t): tE, omega = (t, s) / (t, t); xE, rE updates.
// part: G partials of sum w dphi, G of (t, s), G of (t, t).
template <bool CG>
__device__ __forceinline__ void fin_omega(KrylovScalars *ks, const double *part, int G) {
  const double wdp = sum_partials_t<CG>(part, G);
  const double ts = sum_partials_t<CG>(part + G, G);
  const double tt = sum_partials_t<CG>(part + 2 * G, G);
  if (threadIdx.x == 0) {
    ks->tE = ks->strain ? ks->sE : ks->s3 * wdp;
    const double tst = ts + ks->tE * ks->sE;
    const double ttt = tt + ks->tE * ks->tE;
    ks->omega = ttt > 0.0 ? tst / ttt : 0.0;
    ks->xE += ks->alpha * ks->pE + ks->omega * ks->sE;
    ks->rE = ks->sE - ks->omega * ks->tE;
  }
}

// after x += alpha p + omega s, r = s - omega t: convergence test and the next iteration's
// beta (rho_{k+1} from the fused dot).  part: G partials of |r|^2, then G of (rhat, r).
template <bool CG>
__device__ __forceinline__ void fin_conv(KrylovScalars *ks, const double *part, int G) {
  const double rr = sum_partials_t<CG>(part, G);
  const double rhr = sum_partials_t<CG>(part + G, G);
  if (threadIdx.x == 0) {
    ks->iters += 1;
    const double rn2 = rr + ks->rE * ks->rE;
    ks->rn2 = rn2;
    if (rn2 <= fmax(ks->tol2 * ks->bn2, ks->atol2)) {
      ks->done = 1;
      ks->status = 0;
      return;
    }
    if (ks->omega == 0.0) {
      ks->done = 1;
      ks->status = 2;
      return;
    }
    if (ks->iters >= ks->maxit) {
      ks->done = 1;
      ks->status = 1;
      return;
    }
    const double rho_new = ks->fault_rho0 ? 0.0 : rhr + ks->rhE * ks->rE;
    if (rho_new == 0.0) {
      ks->done = 1;
      ks->status = 2;
      return;
    }
    ks->beta = (rho_new / ks->rho) * (ks->alpha / ks->omega);
    ks->rho = rho_new;
    ks->pE = ks->rE + ks->beta * (ks->pE - ks->omega * ks->vE);
  }
}

// after apply(s -> t) in a float32 chunk: the omega update of fin_omega and the convergence
// test of fin_conv in one step, before r = s - omega t exists as a vector.  With the field
// dots of this apply's epilogue (part: G partials each of sum w dphi, (t, s), (t, t),
// (rhat, s), (rhat, t), (s, s)) the field parts of |r|^2 and (rhat, r) are
//   |r|^2 = (s, s) - 2 omega (t, s) + omega^2 (t, t),   (rhat, r) = (rhat, s) - omega (rhat, t)
// (the float32 run's convergence threshold is far above their rounding).  The vector update
// is left pending; the next x-forward pass or the chunk's closing k_kx_finish applies it.
template <bool CG>
__device__ __forceinline__ void fin_omega_conv(KrylovScalars *ks, const double *part, int G) {
  const double wdp = sum_partials_t<CG>(part, G);
  const double ts = sum_partials_t<CG>(part + G, G);
  const double tt = sum_partials_t<CG>(part + 2 * G, G);
  const double rs = sum_partials_t<CG>(part + 3 * G, G);
  const double rt = sum_partials_t<CG>(part + 4 * G, G);
  const double ss = sum_partials_t<CG>(part + 5 * G, G);
  if (threadIdx.x == 0) {
    ks->tE = ks->strain ? ks->sE : ks->s3 * wdp;
    const double tst = ts + ks->tE * ks->sE;
    const double ttt = tt + ks->tE * ks->tE;
    const double om = ttt > 0.0 ? tst / ttt : 0.0;
    ks->omega = om;
    ks->xE += ks->alpha * ks->pE + om * ks->sE;
    ks->rE = ks->sE - om * ks->tE;
    ks->pending = 1;
    const double rr = fmax(ss - 2.0 * om * ts + om * om * tt, 0.0);
    const double rhr = rs - om * rt;
    ks->iters += 1;
    const double rn2 = rr + ks->rE * ks->rE;
    ks->rn2 = rn2;
    if (rn2 <= fmax(ks->tol2 * ks->bn2, ks->atol2)) {
      ks->done = 1;
      ks->status = 0;
      return;
    }
    if (om == 0.0) {
      ks->done = 1;
      ks->status = 2;
      return;
    }
    if (ks->iters >= ks->maxit) {
      ks->done = 1;
      ks->status = 1;
      return;
    }
    const double rho_new = ks->fault_rho0 ? 0.0 : rhr + ks->rhE * ks->rE;
    if (rho_new == 0.0) {
      ks->done = 1;
      ks->status = 2;
      return;
    }
    ks->beta = (rho_new / ks->rho) * (ks->alpha / om);
    ks->rho = rho_new;
    ks->pE = ks->rE + ks->beta * (ks->pE - om * ks->vE);
  }
}
