"""FP64 CPU oracle for the nuclear-structure DMRG hot path.

TEST INFRASTRUCTURE.  Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import or run anything in this package.  The CUDA library and its
Python binding never import it, and it imports nothing from them; the two share only the
seeded input generator ``gen``.

Contents and pins (each checked by a ``-m "not gpu"`` test):
* ``hamiltonian``: Eq. (1) in the m-scheme determinant basis, dense exact
  diagonalization.  Pinned by the two-particle spectra (they equal the J-coupled matrix
  elements plus single-particle energies), the seniority closed form of a single-j
  pairing Hamiltonian, J-multiplet containment across 2M sectors, the one-body closed
  form, Hermiticity, and the dimension integers quoted for the pf shell.
* ``mpo``: the normal / complementary operator partition of H at every bond.  Pinned by
  brute force: sum_k L_k R_k rebuilt on the full Fock space of small chains equals H from
  Jordan-Wigner matrices, at every bond, in both operator modes.
* ``dmrg``: two-site DMRG.  Pinned by full-M runs reproducing exact diagonalization,
  the variational bound, energies non-increasing in M, Hermiticity of H_eff,
  H_eff on exact states, and truncation error -> 0 at full M.  Its dynamic block state
  selection is pinned by brute force on singular values of the wave-function blocks,
  by its reductions to the fixed-M rule, and by the truncation bound along sweeps.
* ``entropy``: two-orbital density matrix of the dot orbitals and the one- and
  two-orbital entropies; every pair from the written-out state.  Pinned by the exact
  ground state in the determinant basis (occupations, pair occupations, the hopping
  element with determinant signs, for neighbours and across strings) and by equal
  entropies of time-reversed orbitals.
* ``ordering``: chain order from the mutual information (Fiedler vector of the graph
  Laplacian).  Pinned by the path graph's closed form, recovery of a hidden chain, the
  variational property, and brute force over all orders of a small case.
* ``extrapolate``: least-squares E(M) fits.  Pinned by exact model data, the normal
  equations, an independent exponent scan and equivariance under shift and scale.
"""
