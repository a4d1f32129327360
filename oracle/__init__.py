"""FP64 CPU oracle for compressive phase-contrast tomography.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only the test-suite, the smoke check of ``__graft_entry__`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA
library (no kernels, headers, tables or helpers); both sides only share the
seeded input generators, which hold none of the method's arithmetic.

Modules
-------
``nufft``     the Fourier-slice Radon transform and its adjoint, twice: as the
              exact direct non-uniform DFT and as the Kaiser-Bessel gridding
              approximation that the GPU path implements
              (section "fast radon transform").
``ring``      the cubic ring-artifact filter used inside the constraint of the
              L1 problem (section "Introduction", filter / polynomial
              subtraction).
``spgl1``     the SPGL1 Pareto-root-finding basis-pursuit solver applied to
              filter(Radon) (section "Introduction", the L1 problem).
``analytic``  closed forms used as pins: parallel projections of disks.
``unet``      the convolutional denoiser of the learned warm start (no
              counterpart in the paper): forward pass and hand-written
              backward pass in FP64.
``synthesis`` the horizontal finite-difference synthesis operator of the
              analysis-l1 variant (u = C z, its adjoint and its inverse).

Parity status of every function is listed in its module header.
"""
