// Argument blocks of the kernels outside the operator apply (kernels_pw.cu): the dissipated-
// energy constraint (launched by linearize under energy control) and the J-integral
// post-process (launched by rve_j_integral).
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

// Per-frequency operators on the forward half spectra of the float64 residual layout
// [ch][z position][y position][kx] (kx natural; y and z positions digit-reversed:
// ky = yrev[position], kz = zrev[position]).
struct SpecOpArgs {
  Geo g;
  cpx<double> *spec;
  const short *yrev, *zrev;  // zrev unused in 2D
  double inv_n;
};

// Pointwise parts of the dissipated energy int G_c gamma_f and its derivative.
struct EnergyArgs {
  Geo g;
  const double *phi;
  const uint8_t *mat;
  PhaseTab ph;
  double ell;
  double *buf;   // m channels of n doubles (gradient / flux / divergence work space)
  double *part;  // 2 * gridDim.x partials: dissipated energy, |w|^2
};
