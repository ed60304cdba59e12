// Compile-time line length 128: apply passes of fft_passes.cuh (see there).
#include "fft_passes.cuh"
#define RVE_NL 128
#include "fft_inst_ct.cuh"
