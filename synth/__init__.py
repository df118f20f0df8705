"""Seeded synthetic inputs (no arithmetic of the embedded-ERI method)."""
from .lattice import (BATCH_MESHES, CONFIGS, counter_key, counter_normals, batch_specs, complex_supercell_orbitals, LatticeSpec, bloch_orbitals, cell_vectors, dmet_structured_orbitals,
                      fourier_L, make_L, make_L_pairs, make_problem, min_image_norm, phases, real_space_B, spec_with,
                      supercell_orbitals, real_space_fock, fock_k, embedding_density, mean_field_hamiltonian,
                      mean_field_density, lo_rotation, GridSpec, cell_grid_points, ao_supercell, shift_cells,
                      pair_densities_k, grid_orbitals)
