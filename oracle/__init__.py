"""FP64 CPU oracle for the SARA-SDMM imaging method (test infrastructure only).

This package is a plain, slow, obviously correct restatement of what the
method computes, written from the paper's Sections 2-3 (problems (2)-(3),
the splitting (6), the proximity operator definition (7) and Algorithm 1),
in float64 with NumPy/SciPy primitives (FFT, sparse mat-vec, polynomial
roots).  It shares no code with the CUDA library and imports nothing from it.

Only the test suite, the smoke check and the CPU-baseline leg of the
benchmark may import it.  The product path never routes through it.

Modules:
  kaiser_bessel  KB interpolation kernel and its Fourier transform
  nudft          exact non-uniform DFT (pin for the NUFFT only)
  nufft          Phi = G F Z S and its adjoint (the measurement operator)
  daubechies     Db1..Db8 filters by spectral factorisation
  dwt            periodic 2D orthonormal wavelet transform
  sara           the SARA dictionary Psi = [Dirac, Db1..Db8] / 3
  prox           closed-form proximity operators
  cg             conjugate gradient on the SDMM normal operator
  sdmm           Algorithm 1 and the SARA reweighting loop
  simulate       input-SNR noise rule, epsilon rule, SNR metric

Parity status: every function here is pinned by a test under tests/ against
a closed form, a brute-force computation, a certificate or a library
routine.  The SARA weight rule and the reweighting loop are pinned as a
majorise-minimise descent at fixed delta; the delta schedule itself
(sdmm.delta_schedule) is a reading the paper does not fix: "parity unpinned"
for it.
"""
