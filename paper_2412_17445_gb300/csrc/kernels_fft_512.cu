// Compile-time line length 512: apply passes of fft_passes.cuh (see there).
#include "fft_passes.cuh"
#define RVE_NL 512
#include "fft_inst_ct.cuh"
