// Compile-time line length 64: apply passes of fft_passes.cuh (see there).
#include "fft_passes.cuh"
#define RVE_NL 64
#include "fft_inst_ct.cuh"
