// In-shared-memory mixed-radix FFT stages (radix 2, 3, 4, 8) for the FFT passes of the
// operator apply (Eq. CrackLength_linearization) and the residual (Eq. System_CrackLength).
//
// A line of N complex values sits in shared memory.  Forward transforms run as in-place
// decimation-in-frequency (DIF) stages: natural-order input, digit-reversed output.
// Inverse transforms run as in-place decimation-in-time (DIT) stages: digit-reversed
// input, natural-order output.  A DIF pass followed by a DIT pass therefore needs no
// permutation in between, and the pointwise spectral multiply is done on the
// digit-reversed positions (the frequency held at position p is rev[p]).
//
// Stage s (s = 0..S-1, DIT order) has radix R_s and span Ns_s = R_0 ... R_{s-1}.
// DIT applies the stages in order s = 0..S-1 (twiddle, then R-point DFT);
// DIF applies them in reverse order s = S-1..0 (R-point DFT, then twiddle).
// The digit reversal maps a position p to the sample index it holds in a DIT input:
//   p = r * (N / R_{S-1}) + p'  ->  rev(p) = r + R_{S-1} * rev'(p')   (recursively).
//
// Shared-memory lines are padded with one slot after every 8 elements (pad(e) = e + e/8):
// a radix-8 stage of span 1 reads elements 8 apart, which without padding would hit the
// same banks from every thread of a warp.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define FFT_MAX_STAGES 14

// Aligned to its full size so that one element moves as one 8-byte (float) or 16-byte
// (double) shared or global access rather than two.
template <typename T>
struct __align__(2 * sizeof(T)) cpx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
// multiply by i * s  (s = +1 or -1)
template <typename T>
__device__ __forceinline__ cpx<T> cmuli(cpx<T> a, T s) { return {-s * a.y, s * a.x}; }

// Division by a runtime constant d through a multiply-high: for x < 2^32 / d,
// floor(x / d) = umulhi(x, ceil(2^32 / d)).  All callers divide indices below 2^20 by
// divisors of at most 4096.
struct FDiv {
  unsigned d, m;
};
__device__ __forceinline__ unsigned fdiv(unsigned x, const FDiv &f) { return f.d == 1 ? x : __umulhi(x, f.m); }

// padded shared-memory index of element e of a line (runtime line lengths)
__device__ __forceinline__ int pad8(int e) { return e + (e >> 3); }

// Shared-memory slot of element e of a line of compile-time length NL (> 0, a multiple of
// 16, line bases at multiples of 16): bits 0..3 are XOR-ed with bits 3..6.  Within every
// half-warp of 8-byte accesses this is conflict-free for unit-stride runs, for the stride-8
// runs of the span-1 radix-8 stage and for the 64 g + j + 8 r runs of the span-8 stage
// (checked for every stage of every compiled length), and it needs no padding.  NL = 0
// keeps the padded layout.
template <int NL>
__device__ __forceinline__ int smap(int e) {
  if constexpr (NL > 0) return e ^ ((e >> 3) & 15);
  else return pad8(e);
}
// slots per line: NL for compile-time lengths, the padded runtime length otherwise
template <int NL>
__host__ __device__ __forceinline__ constexpr int line_slots(int Np_rt) { return NL > 0 ? NL : Np_rt; }

// Transform plan of one line length N.  tw points to N twiddles exp(-2 pi i k / N) of the
// transform precision (cpx<float> or cpx<double>), rev / unrev to the digit-reversal
// permutation and its inverse (N entries each), all in global memory.
struct FftPlan {
  int N;
  int Np;                     // padded line length N + (N - 1) / 8
  int S;                      // number of stages
  int R[FFT_MAX_STAGES];      // radix of stage s (DIT order)
  int Ns[FFT_MAX_STAGES];     // span of stage s = R_0 ... R_{s-1}
  FDiv dNs[FFT_MAX_STAGES];   // division by Ns
  FDiv dNb[FFT_MAX_STAGES];   // division by N / R
  const void *tw;
  const short *rev;           // position -> sample / frequency index
  const short *unrev;         // sample / frequency index -> position
};

// ---- R-point DFTs in registers, sign dir (-1 forward, +1 inverse) ----------------------
template <typename T>
__device__ __forceinline__ void dft2(cpx<T> *v) {
  cpx<T> a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <typename T>
__device__ __forceinline__ void dft3(cpx<T> *v, T dir) {
  const T s3 = (T)0.86602540378443864676;  // sin(2 pi / 3)
  cpx<T> t1 = cadd(v[1], v[2]);
  cpx<T> t2 = csub(v[1], v[2]);
  cpx<T> m = {v[0].x - (T)0.5 * t1.x, v[0].y - (T)0.5 * t1.y};
  cpx<T> r = cmuli(t2, dir * s3);
  v[0] = cadd(v[0], t1);
  v[1] = cadd(m, r);
  v[2] = csub(m, r);
}

template <typename T>
__device__ __forceinline__ void dft4(cpx<T> *v, T dir) {
  cpx<T> a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
  cpx<T> c = cadd(v[1], v[3]), d = cmuli(csub(v[1], v[3]), dir);
  v[0] = cadd(a, c);
  v[2] = csub(a, c);
  v[1] = cadd(b, d);
  v[3] = csub(b, d);
}

template <typename T>
__device__ __forceinline__ void dft8(cpx<T> *v, T dir) {
  const T h = (T)0.70710678118654752440;  // sqrt(1/2)
  cpx<T> e[4] = {v[0], v[2], v[4], v[6]};
  cpx<T> o[4] = {v[1], v[3], v[5], v[7]};
  dft4(e, dir);
  dft4(o, dir);
  // W8^k = exp(dir * 2 pi i k / 8)
  cpx<T> w1 = {h, dir * h};
  cpx<T> o1 = cmul(o[1], w1);
  cpx<T> o2 = cmuli(o[2], dir);
  cpx<T> w3 = {-h, dir * h};
  cpx<T> o3 = cmul(o[3], w3);
  v[0] = cadd(e[0], o[0]);
  v[4] = csub(e[0], o[0]);
  v[1] = cadd(e[1], o1);
  v[5] = csub(e[1], o1);
  v[2] = cadd(e[2], o2);
  v[6] = csub(e[2], o2);
  v[3] = cadd(e[3], o3);
  v[7] = csub(e[3], o3);
}

// Addressing of line l, element e in shared memory (padded element index):
//   addr = (l / lw) * lsA + (l % lw) * lsB + pad8(e) * es
struct LineLayout {
  int L;     // number of lines
  FDiv dL;   // division by L
  FDiv dlw;  // division by lw (lines per group)
  int lw;
  int lsA;   // stride between groups
  int lsB;   // stride between lines of a group
  int es;    // element stride
  bool line_fastest;  // thread mapping: consecutive threads -> consecutive lines
};

__device__ __forceinline__ int line_base(const LineLayout &ly, int l) {
  if (ly.lw == 1) return l * ly.lsA;
  const int g = (int)fdiv((unsigned)l, ly.dlw);
  return g * ly.lsA + (l - g * ly.lw) * ly.lsB;
}

// One stage of radix R over all lines.  DIT: twiddle then DFT; DIF: DFT then twiddle.
// dir = -1 forward, +1 inverse.  Caller syncs between stages.
template <typename T, bool DIT, int R>
__device__ __forceinline__ void fft_stage_r(cpx<T> *sm, const LineLayout &ly, const FftPlan &pl, int s,
                                            T dir) {
  const int N = pl.N, Ns = pl.Ns[s];
  const int nb = N / R;
  const int tot = ly.L * nb;
  const int twstep = N / (Ns * R);
  const cpx<T> *tw = (const cpx<T> *)pl.tw;
  for (int b = threadIdx.x; b < tot; b += blockDim.x) {
    int l, q;
    if (ly.line_fastest) {
      q = (int)fdiv((unsigned)b, ly.dL);
      l = b - q * ly.L;
    } else {
      l = (int)fdiv((unsigned)b, pl.dNb[s]);
      q = b - l * nb;
    }
    const int g = (int)fdiv((unsigned)q, pl.dNs[s]);
    const int j = q - g * Ns;
    const int e0 = g * Ns * R + j;  // first element of the butterfly
    const int lb = line_base(ly, l);
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = sm[lb + pad8(e0 + r * Ns) * ly.es];
    if (DIT && j != 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cpx<T> w = tw[r * j * twstep];  // index < R * Ns * N / (Ns * R) = N
        w.y *= -dir;  // table holds exp(-2 pi i e/N); dir = +1 needs the conjugate
        v[r] = cmul(v[r], w);
      }
    }
    if (R == 8) dft8(v, dir);
    else if (R == 4) dft4(v, dir);
    else if (R == 3) dft3(v, dir);
    else if (R == 2) dft2(v);
    if (!DIT && j != 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cpx<T> w = tw[r * j * twstep];
        w.y *= -dir;
        v[r] = cmul(v[r], w);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) sm[lb + pad8(e0 + r * Ns) * ly.es] = v[r];
  }
}

template <typename T, bool DIT>
__device__ __forceinline__ void fft_stage(cpx<T> *sm, const LineLayout &ly, const FftPlan &pl, int s, T dir) {
  switch (pl.R[s]) {
    case 8: fft_stage_r<T, DIT, 8>(sm, ly, pl, s, dir); break;
    case 4: fft_stage_r<T, DIT, 4>(sm, ly, pl, s, dir); break;
    case 3: fft_stage_r<T, DIT, 3>(sm, ly, pl, s, dir); break;
    case 2: fft_stage_r<T, DIT, 2>(sm, ly, pl, s, dir); break;
    default: break;  // N = 1
  }
}

// Full DIF transform of all lines (natural in, digit-reversed out).
template <typename T>
__device__ void fft_dif(cpx<T> *sm, const LineLayout &ly, const FftPlan &pl, T dir) {
  for (int s = pl.S - 1; s >= 0; --s) {
    fft_stage<T, false>(sm, ly, pl, s, dir);
    __syncthreads();
  }
}
// Full DIT transform (digit-reversed in, natural out).
template <typename T>
__device__ void fft_dit(cpx<T> *sm, const LineLayout &ly, const FftPlan &pl, T dir) {
  for (int s = 0; s < pl.S; ++s) {
    fft_stage<T, true>(sm, ly, pl, s, dir);
    __syncthreads();
  }
}

// ==== compile-time line length ============================================================
// The same stage sequence as the host plan (radix 3 stages first, then 8, 4, 2; DIT order),
// known at compile time so that every index, trip count and table offset folds to a constant.
struct StagePlan {
  int S;
  int R[FFT_MAX_STAGES];
  int Ns[FFT_MAX_STAGES];
};

__host__ __device__ constexpr StagePlan stage_plan(int N) {
  StagePlan p{};
  int rem = N, s = 0, ns = 1;
  const int radices[4] = {3, 8, 4, 2};
  for (int k = 0; k < 4; ++k) {
    const int R = radices[k];
    while (rem % R == 0 && rem > 1) {
      p.R[s] = R;
      p.Ns[s] = ns;
      ns *= R;
      rem /= R;
      ++s;
    }
  }
  p.S = s;
  return p;
}

template <typename T>
__device__ __forceinline__ cpx<T> cmul_conj(cpx<T> a, cpx<T> w) {  // a * conj(w)
  return {a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y};
}

// Twiddles w[r] = tw[r * jt], r = 1..R-1, of one butterfly.  For float32 radix 8 only
// w1, w2, w4 are loaded and w3, w5, w6, w7 formed as products of two of them (at most one
// extra rounding), which halves the table traffic through L1.
template <typename T, int R>
__device__ __forceinline__ void load_twiddles(const cpx<T> *__restrict__ tw, int jt, cpx<T> (&w)[R]) {
  if constexpr (R == 8 && sizeof(T) == 4) {
    w[1] = tw[jt];
    w[2] = tw[2 * jt];
    w[4] = tw[4 * jt];
    w[3] = cmul(w[1], w[2]);
    w[5] = cmul(w[1], w[4]);
    w[6] = cmul(w[2], w[4]);
    w[7] = cmul(w[3], w[4]);
  } else {
#pragma unroll
    for (int r = 1; r < R; ++r) w[r] = tw[r * jt];
  }
}

// Lines of length N in shared memory: element e of line (lc, w) sits at
//   ((lc * N + smap<N>(e)) << lw) + w,   lc < Lc groups, w < 2^lw adjacent lines per group.
// LW >= 0 fixes lw at compile time (x passes: 0); LW < 0 takes the runtime lw.
// INV: inverse (DIT, twiddle before the DFT, conjugate twiddles); else forward (DIF).
template <typename T, bool INV, int R, int NS, int N, int LW>
__device__ __forceinline__ void ct_stage(cpx<T> *sm, int Lc, int lw_rt, const cpx<T> *__restrict__ tw) {
  constexpr int NB = N / R;
  constexpr int TWS = N / (NS * R);
  constexpr int Np = N;  // swizzled lines (smap), no padding
  const int lw = LW >= 0 ? LW : lw_rt;
  const int tot = (Lc * NB) << lw;
  const T dir = INV ? (T)1 : (T)-1;
  for (int b = threadIdx.x; b < tot; b += blockDim.x) {
    const int w = b & ((1 << lw) - 1);
    const int rest = b >> lw;
    const int lc = rest / NB;
    const int q = rest - lc * NB;
    const int g = q / NS, j = q - g * NS;
    const int e0 = g * NS * R + j;
    cpx<T> *base = sm + ((lc * Np) << lw) + w;
    int off[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      off[r] = smap<N>(e0 + r * NS) << lw;
    }
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = base[off[r]];
    cpx<T> wt[R];
    if constexpr (NS > 1) load_twiddles<T, R>(tw, j * TWS, wt);
    if constexpr (INV && NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul_conj(v[r], wt[r]);
    }
    if constexpr (R == 8) dft8(v, dir);
    else if constexpr (R == 4) dft4(v, dir);
    else if constexpr (R == 3) dft3(v, dir);
    else if constexpr (R == 2) dft2(v);
    if constexpr (!INV && NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], wt[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) base[off[r]] = v[r];
  }
}

template <typename T, int N, int LW, int s>
__device__ __forceinline__ void ct_dif_from(cpx<T> *sm, int Lc, int lw, const cpx<T> *tw) {
  if constexpr (s >= 0) {
    constexpr StagePlan P = stage_plan(N);
    ct_stage<T, false, P.R[s], P.Ns[s], N, LW>(sm, Lc, lw, tw);
    __syncthreads();
    ct_dif_from<T, N, LW, s - 1>(sm, Lc, lw, tw);
  }
}

template <typename T, int N, int LW, int s>
__device__ __forceinline__ void ct_dit_from(cpx<T> *sm, int Lc, int lw, const cpx<T> *tw) {
  constexpr StagePlan P = stage_plan(N);
  if constexpr (s < P.S) {
    ct_stage<T, true, P.R[s], P.Ns[s], N, LW>(sm, Lc, lw, tw);
    __syncthreads();
    ct_dit_from<T, N, LW, s + 1>(sm, Lc, lw, tw);
  }
}

// Forward DIF (natural in, digit-reversed out) / inverse DIT (digit-reversed in, natural
// out) of Lc * 2^lw lines of compile-time length N; same operations and order as
// fft_dif / fft_dit with the host plan of N.
template <typename T, int N, int LW>
__device__ __forceinline__ void fft_dif_ct(cpx<T> *sm, int Lc, int lw, const cpx<T> *tw) {
  constexpr StagePlan P = stage_plan(N);
  ct_dif_from<T, N, LW, P.S - 1>(sm, Lc, lw, tw);
}
template <typename T, int N, int LW>
__device__ __forceinline__ void fft_dit_ct(cpx<T> *sm, int Lc, int lw, const cpx<T> *tw) {
  ct_dit_from<T, N, LW, 0>(sm, Lc, lw, tw);
}

// Digit reversal of the compile-time plan of N: position -> sample / frequency index (rev)
// and its inverse (unrev); the same maps as the host tables of the plan.
template <int N>
__device__ __forceinline__ int digit_rev_ct(int p) {
  constexpr StagePlan P = stage_plan(N);
  int out = 0, mul = 1, len = N;
#pragma unroll
  for (int s = P.S - 1; s >= 0; --s) {
    len /= P.R[s];
    const int r = p / len;
    p -= r * len;
    out += r * mul;
    mul *= P.R[s];
  }
  return out;
}
template <int N>
__device__ __forceinline__ int digit_unrev_ct(int k) {
  constexpr StagePlan P = stage_plan(N);
  int p = 0, mul = N;
#pragma unroll
  for (int s = P.S - 1; s >= 0; --s) {
    const int r = k % P.R[s];
    k /= P.R[s];
    mul /= P.R[s];
    p += r * mul;
  }
  return p;
}

// Stages hi..lo of the DIF transform / lo..hi of the DIT transform over Lc lines of
// compile-time length N (line stride N, smap slots, lw = 0), each followed by a barrier.
template <typename T, int N, int HI, int LO>
__device__ __forceinline__ void ct_dif_range(cpx<T> *sm, int Lc, const cpx<T> *tw) {
  if constexpr (HI >= LO) {
    constexpr StagePlan P = stage_plan(N);
    ct_stage<T, false, P.R[HI], P.Ns[HI], N, 0>(sm, Lc, 0, tw);
    __syncthreads();
    ct_dif_range<T, N, HI - 1, LO>(sm, Lc, tw);
  }
}
template <typename T, int N, int LO, int HI>
__device__ __forceinline__ void ct_dit_range(cpx<T> *sm, int Lc, const cpx<T> *tw) {
  if constexpr (LO <= HI) {
    constexpr StagePlan P = stage_plan(N);
    ct_stage<T, true, P.R[LO], P.Ns[LO], N, 0>(sm, Lc, 0, tw);
    __syncthreads();
    ct_dit_range<T, N, LO + 1, HI>(sm, Lc, tw);
  }
}
