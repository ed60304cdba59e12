// Explicit instantiations of the apply passes for the compile-time line length RVE_NL.
// 2D (m = 3) at every length; 3D (m = 6) at the lengths of the 3D grids (<= 128).  RVE_NL is a
// multiple of 16 (the shared-memory swizzle of fft.cuh permutes within aligned groups of 16).
// (2D runs only the fused column pass, mode 1.)
#define INST_CT2(T)                                                                  \
  template __global__ void k_xfwd_apply<T, 3, RVE_NL, 0, -1>(const __grid_constant__ ApplyGroup<T>, FftPlan, int);   \
  template __global__ void k_xinv_apply<T, 3, RVE_NL, 0, -1>(const __grid_constant__ ApplyGroup<T>, FftPlan, int);   \
  template __global__ void k_col<T, 3, 1, RVE_NL>(const __grid_constant__ ColGroup<T>);
#define INST_CT3(T)                                                                  \
  template __global__ void k_xfwd_apply<T, 6, RVE_NL, 0, -1>(const __grid_constant__ ApplyGroup<T>, FftPlan, int);   \
  template __global__ void k_xinv_apply<T, 6, RVE_NL, 0, -1>(const __grid_constant__ ApplyGroup<T>, FftPlan, int);   \
  template __global__ void k_col<T, 6, 0, RVE_NL>(const __grid_constant__ ColGroup<T>);                       \
  template __global__ void k_col<T, 6, 1, RVE_NL>(const __grid_constant__ ColGroup<T>);                       \
  template __global__ void k_col<T, 6, 2, RVE_NL>(const __grid_constant__ ColGroup<T>);
INST_CT2(float)
// float32 2D passes with the row pairs per block (1 or 2) and the fused prologue / epilogue
// mode fixed at compile time: x-forward modes 0 (plain), 1 (p update), 2 (s update),
// 4 (projection), 5 (pending x / r update, then p update); x-inverse modes 0 (plain), 1 (dot
// with rhat), 2 (dots with s), 3 (projection), 6 (the five dots of the merged update)
#define INST_SPEC(PC)                                                                                    \
  template __global__ void k_xfwd_apply<float, 3, RVE_NL, PC, 0>(const __grid_constant__ ApplyGroup<float>, FftPlan, int); \
  template __global__ void k_xfwd_apply<float, 3, RVE_NL, PC, 1>(const __grid_constant__ ApplyGroup<float>, FftPlan, int); \
  template __global__ void k_xfwd_apply<float, 3, RVE_NL, PC, 2>(const __grid_constant__ ApplyGroup<float>, FftPlan, int); \
  template __global__ void k_xfwd_apply<float, 3, RVE_NL, PC, 4>(const __grid_constant__ ApplyGroup<float>, FftPlan, int); \
  template __global__ void k_xfwd_apply<float, 3, RVE_NL, PC, 5>(const __grid_constant__ ApplyGroup<float>, FftPlan, int); \
  template __global__ void k_xinv_apply<float, 3, RVE_NL, PC, 0>(const __grid_constant__ ApplyGroup<float>, FftPlan, int); \
  template __global__ void k_xinv_apply<float, 3, RVE_NL, PC, 1>(const __grid_constant__ ApplyGroup<float>, FftPlan, int); \
  template __global__ void k_xinv_apply<float, 3, RVE_NL, PC, 2>(const __grid_constant__ ApplyGroup<float>, FftPlan, int); \
  template __global__ void k_xinv_apply<float, 3, RVE_NL, PC, 3>(const __grid_constant__ ApplyGroup<float>, FftPlan, int); \
  template __global__ void k_xinv_apply<float, 3, RVE_NL, PC, 6>(const __grid_constant__ ApplyGroup<float>, FftPlan, int);
INST_SPEC(1)
INST_SPEC(2)
// the fused column pass runs at the power-of-two lengths (its span-1 stage is radix 8)
#if (RVE_NL & (RVE_NL - 1)) == 0
template __global__ void k_col_fused2d<RVE_NL, 2048 / RVE_NL>(const __grid_constant__ ColGroup<float>);
template __global__ void k_col_fused2d<RVE_NL, 1024 / RVE_NL>(const __grid_constant__ ColGroup<float>);
#if RVE_NL <= 512
template __global__ void k_col_fused2d<RVE_NL, 512 / RVE_NL>(const __grid_constant__ ColGroup<float>);
#endif
#endif
INST_CT2(double)
#if RVE_NL <= 128
INST_CT3(float)
INST_CT3(double)
#endif
