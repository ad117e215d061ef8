"""Plain CPU FP64 oracle for the flat-layer inverse-acoustics method
(Bakushinsky & Leonov, arXiv 1911.10487).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the tests, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it.
The product path (the CUDA library and its Python binding) never imports,
calls or links anything here, and this package imports nothing from the
product.

It is written for a reader checking it against the paper by eye: NumPy/SciPy
in float64/complex128, every step in the order the paper states it, no
blocking, fusion or reordering.  Each function cites the passage it follows.

Modules
  grid       discrete conventions (periodic horizontal grid, X/Y planes, wavenumbers)
  kernel     Weyl closed form of the horizontal Fourier transform of G (Sec. 2, eq. 5)
  operators  discrete X->Y and X->X operators (eq. 5), FFT and explicit-DFT forms
  forward    forward data generator: Algorithm 1 (eq. 6-7), GMRES, dense LU, Born
  inverse    Algorithm 2 (eq. 8-9, step 3) with Tikhonov + discrepancy principle
  adjoint    reverse-mode derivative of Algorithm 2 at fixed alpha
  metrics    relative L2 errors, Delta_L2(z) (Sec. 5.3)
"""
