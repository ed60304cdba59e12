// Compile-time line length 256: apply passes of fft_passes.cuh (see there).
#include "fft_passes.cuh"
#define RVE_NL 256
#include "fft_inst_ct.cuh"
