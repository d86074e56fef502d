"""CPU oracle for the linear-response hot path of arXiv:2505.02319.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 NumPy
restatement of what the method computes.  It is imported only by ``tests/``,
by ``__graft_entry__.smoke()`` and by the CPU-baseline / reference legs of
``bench.py``; the GPU library never imports, calls or links it, and it shares
no code with the CUDA path.

Where the method reaches, up to rounding, a result with a plain definition
the oracle is that definition written out:
  * Fourier transforms F, F^-1 (eq. fft_ifft) as naive separable DFT sums;
  * the Hamiltonian (eq. Hamiltonian, k-form of Sec. 4.1.1) as a dense matrix,
    diagonalised densely (NumPy eigh) for the ground state;
  * chi0 (eqs. chi0, delta_f, delta_phi_P; k-form eq. kchi0) with the
    Sternheimer equations (eq. discretised_sternheimer) solved exactly by the
    pseudo-inverse A_n^+ = Phi_perp D_n^-1 Phi_perp^H (proof of Lemma cgtol_E);
  * the dielectric adjoint E = 1 - chi0 K (eq. op_discretised), and the Dyson
    solution by a dense solve (tiny grids) or GMRES with exact products;
  * Algorithm 1 (inexact GMRES) with the CG tolerances of Table strategies /
    Table strategies_k, emulated with a plain NumPy CG, for strategy tests.

Readings where the paper is silent or garbled are stated in the docstrings
of the functions that take them.

Parity unpinned: nothing in this package.  Every function is pinned by a
``-m "not gpu"`` test in tests/test_oracle_*.py.
"""
