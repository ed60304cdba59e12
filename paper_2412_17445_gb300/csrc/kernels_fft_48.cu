// Compile-time line length 48 = 3 x 16: apply passes of fft_passes.cuh (see there).
#include "fft_passes.cuh"
#define RVE_NL 48
#include "fft_inst_ct.cuh"
