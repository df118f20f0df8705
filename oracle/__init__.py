"""CPU oracle for the embedded-ERI transformation (test infrastructure).

A plain, slow, FP64 restatement of Algorithm 1 of Cui, Zhu & Chan, "Efficient
Implementation of Ab Initio Quantum Embedding in Periodic Systems: Density Matrix
Embedding Theory" (arXiv 1909.08596), section 2.1, and of the embedding one-particle
Hamiltonian of the same section (Eqs. "fock transform" and "fock double counting") and of
the DMET bath construction before it (Eqs. "bath R SVD", "C loemb R" and "C loemb k") and of the
FFTDF variant of Appendix B (Algorithm 2, Eq. "FFTDF"),
together with brute-force real-space supercell transformations and the checks the tests use.

This package is test infrastructure. Only the tests, the smoke entry point and the
benchmark's CPU-baseline leg may import it. It shares no code with the CUDA library
(no kernels, headers, index tables or packing helpers) and imports nothing from it;
the product path never calls it.

Parity status: every function here is pinned by tests that do not go through the
function itself (brute force over the supercell, a hand-derived worked example,
closed forms, symmetries, positivity and unitary invariance); see tests/test_oracle_pins.py,
tests/test_oracle_fock_pins.py, tests/test_oracle_bath_pins.py and tests/test_oracle_fftdf_pins.py.
"""
from .mesh import k_add, k_index, k_neg, k_triplet
from .alg1 import embedded_3idx, embedded_eri, embedded_eri_pblocks, eri_entries
from .supercell import (supercell_bath, supercell_density, supercell_eri, supercell_eri_grid, supercell_fock,
                        supercell_matrix)
from .bath import bath_svd, embedding_orbitals, embedding_orbitals_lo, offdiag_density
from .fftdf import coulomb_kernel, embedded_3idx_grid, embedded_eri_fftdf
from .fock import coulomb_exchange, coulomb_exchange_df, embedded_fock, fock_transform
from .checks import orthonormality_error, realness_error, pack_s8, pair_matrix, unpack_s8
from .schedule import schedule
