// Argument blocks of the J-integral post-process (2D): the rotation spectrum kernel and the
// contour sum (kernels_pw.cu), launched by rve_j_integral (rve.cu).
#pragma once
#include "rve_kern.cuh"

// w-hat from the y-forward half spectra of the strain fluctuation (Mandel channels 0..2,
// layout [ch][y position][kx], y positions digit-reversed: ky = yrev[position]); the result
// replaces channel 0, scaled by 1/n for the unnormalised inverse transform.
struct RotArgs {
  Geo g;
  cpx<double> *spec;
  const short *yrev;
  double inv_n;
};

// Rice's J in the x direction over the rectangle of voxel centres (x0, y0)-(x1, y1).
struct JArgs {
  Geo g;
  const double *eps_t;  // Mandel, 3 channels of n
  const double *phi;
  const double *w;      // rotation field, n
  const uint8_t *mat;
  PhaseTab ph;
  double fM[3];
  double E, k_res;
  int isotropic;
  int x0, y0, x1, y1;
  double *out;          // one double
};
