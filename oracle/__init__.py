"""FP64 CPU oracle for the Vanka-smoothed shifted-Laplacian multigrid
preconditioned FGMRES solver of Yovel, He & Treister (arXiv 2511.16808).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the paper's method in numpy/scipy (complex128 throughout).  It
exists to check the CUDA path; the product never imports it.  Only the test
suite, the smoke check of the build entry point and the benchmark's CPU
baseline leg may import or run anything here.  It shares no code with the CUDA
library: the two meet only in the seeded input generators of `workloads`.

Modules
  operator   Eq. (1) discretised on a nodal grid (Section 2.1), the complex
             shift (Eq. shift), and the compact 4th-order stencils
             (Eqs. disc4thCompact, disc4thCompact3D) used by the pins
  transfer   restriction / prolongation (Eqs. biliniearIntergrid,
             bicubicIntergrid, trilin, tricub) and the intergrid schemes
             (Eqs. level1Intergrid, levelDepIntergrid; Section 5.2)
  vanka      patches (Section 3.2), boundary patches and weights
             (Section 3.3), additive Vanka smoother (Eq. smoother), Jacobi
  multigrid  Galerkin hierarchy (Section 3.1), V-cycle (Algorithm 1)
  fgmres     flexible GMRES(m) with right preconditioning (Section 2.3)
  lfa        local Fourier analysis (Section 4, Definitions 2.1-2.3)
  defaults   the paper's damping table (Table relaxParam)

Parity notes: every function names the passage it follows; functions whose
result no test pins against an independent fact say "parity unpinned".
"""
