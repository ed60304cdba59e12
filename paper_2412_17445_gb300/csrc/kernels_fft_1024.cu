// Compile-time line length 1024: apply passes of fft_passes.cuh (see there).
#include "fft_passes.cuh"
#define RVE_NL 1024
#include "fft_inst_ct.cuh"
