"""Plain FP64 CPU oracle for the Generalized Source Method (GSM) solve of a 3D
periodic dielectric composite (Shcherbakov & Tishchenko, arXiv:1501.01752).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code with the CUDA path
(``paper_1501_01752_b300/csrc``); the two meet only through the seeded input
generators in ``paper_1501_01752_b300/workloads.py``, which hold geometry and
random numbers but none of the method's arithmetic.

Everything here is written for clarity, not speed: complex128 numpy, library
primitives (numpy/scipy FFT, LU, least squares, eigenvalues) used as single
steps, and no blocking or fusion beyond what the paper's definitions state.

Modules
-------
coefficients  Fourier images of the permittivity ("Calculation details";
              coefficient array of Eq. 4).
operator      The truncated Eq. 4 operator A = I - G (Delta/eps_b *), the
              Green tensor, the explicit Toeplitz matrix and the FFT form;
              the H-field operator of Eq. 5 in both forms.
solvers       Dense LU, GMRES with modified Gram-Schmidt (Saad), BiCGSTAB.
poles         Resonance model Eq. 6 and the pole fit of Eqs. 7-10.
retrieval     Response xi(kappa), kappa sweeps and the effective tensor.
adjoint       A^H, the gradient of xi with respect to the coefficients and to
              voxel permittivities.

Parity status: every function carries a pin in ``tests/test_oracle_*.py``;
none is "parity unpinned" except where its docstring says so.
"""
