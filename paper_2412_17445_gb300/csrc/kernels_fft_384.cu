// Compile-time line length 384 = 3 x 128: apply passes of fft_passes.cuh (see there).
#include "fft_passes.cuh"
#define RVE_NL 384
#include "fft_inst_ct.cuh"
