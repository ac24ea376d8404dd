"""CPU FP64 oracle for the block-preconditioned VIE-FFT method (arXiv 2501.13512).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package:
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may call it. It shares no code with the CUDA library; the only
module both sides use is the seeded input generator
``paper_2501_13512_gb300.inputs``, which holds none of the method's arithmetic.

Every function is a plain, slow restatement of the passage it cites, in
complex128, using numpy's FFT and dense LU as library primitives.

Discretisation read from Section II.A (Eqs. 1-4): the VIE is written in the
total field E (J = j w eps0 chi E, chi = eps_r - 1), discretised with pulse
basis functions and collocation at voxel centres on the uniform grid:

    (A x)_i = x_i - sum_j K(i - j) chi_j x_j,     b = E_inc,

with K(D) = k0^2 G(D h) h^3 for D != 0 (G the dyadic Green's function of
Eq. 1 built from the scalar g = exp(-jkR)/(4 pi R)) and K(0) = s_self I, the
equivalent-sphere self term. Parity status per function is stated in each
module header.
"""
