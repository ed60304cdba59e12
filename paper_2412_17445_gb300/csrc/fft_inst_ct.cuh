// Explicit instantiations of the apply passes for the compile-time line length RVE_NL.
// 2D (m = 3) at every length; 3D (m = 6) at the lengths of the 3D grids (<= 128).
// (2D runs only the fused column pass, mode 1.)
#define INST_CT2(T)                                                                  \
  template __global__ void k_xfwd_apply<T, 3, RVE_NL>(ApplyArgs<T>, FftPlan, int);   \
  template __global__ void k_xinv_apply<T, 3, RVE_NL>(ApplyArgs<T>, FftPlan, int);   \
  template __global__ void k_col<T, 3, 1, RVE_NL>(ColArgs<T>);
#define INST_CT3(T)                                                                  \
  template __global__ void k_xfwd_apply<T, 6, RVE_NL>(ApplyArgs<T>, FftPlan, int);   \
  template __global__ void k_xinv_apply<T, 6, RVE_NL>(ApplyArgs<T>, FftPlan, int);   \
  template __global__ void k_col<T, 6, 0, RVE_NL>(ColArgs<T>);                       \
  template __global__ void k_col<T, 6, 1, RVE_NL>(ColArgs<T>);                       \
  template __global__ void k_col<T, 6, 2, RVE_NL>(ColArgs<T>);
INST_CT2(float)
template __global__ void k_col_fused2d<RVE_NL, 2048 / RVE_NL>(ColArgs<float>);
template __global__ void k_col_fused2d<RVE_NL, 1024 / RVE_NL>(ColArgs<float>);
#if RVE_NL <= 512
template __global__ void k_col_fused2d<RVE_NL, 512 / RVE_NL>(ColArgs<float>);
#endif
INST_CT2(double)
#if RVE_NL <= 128
INST_CT3(float)
INST_CT3(double)
#endif
