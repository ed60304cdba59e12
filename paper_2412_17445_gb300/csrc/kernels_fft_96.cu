// Compile-time line length 96 = 3 x 32: apply passes of fft_passes.cuh (see there).
#include "fft_passes.cuh"
#define RVE_NL 96
#include "fft_inst_ct.cuh"
