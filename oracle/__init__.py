"""FP64 CPU oracle for the crack-length-controlled phase-field FFT solver (arXiv 2412.17445).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the CUDA
library (no kernels, headers, tables or helpers); the two meet only in the seeded
input generators of ``paper_2412_17445_gb300.microstructure``, which hold none of the
method's arithmetic and which this package does not import either.

The oracle is plain NumPy in float64 and follows the paper's equations in their own
notation, one step at a time:

  fourier.py   frequencies, the Galerkin projection (Eq. GFourier, symmetric reading,
               Willot rotated frequencies of Sec. 3.1), the spectral Laplacian
               (Eq. LinearOpe_Helm) and the crack length (Eqs. CrackLenght,
               newGammaFourier via Parseval)
  material.py  spectral split (Eq. PlusNegPsi), degradation (Eq. gFunct), stress and
               the tangent C (Eq. C_Calc) as a directional derivative
  solver.py    residual F (Eq. System_CrackLength), its linearisation (Eq.
               CrackLength_linearization, Eq. Delta_history), BiCGStab (Sec. 3.2),
               the monolithic Newton loop with crack-length control (Algorithm 2),
               the history update (Eq. history) and the start-up elastic steps
  dense.py     brute-force references used only to pin the oracle: dense DFT,
               dense real-space projector, dense Jacobian, dense-LU Newton

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants or brute force.  Readings of passages where the paper is silent, garbled or
inconsistent are listed in the design notes of the repository and marked
"reading:" in the docstrings here.
"""
