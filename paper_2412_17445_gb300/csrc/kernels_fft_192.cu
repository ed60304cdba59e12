// Compile-time line length 192 = 3 x 64: apply passes of fft_passes.cuh (see there).
#include "fft_passes.cuh"
#define RVE_NL 192
#include "fft_inst_ct.cuh"
