"""Plain, slow FP64 CPU oracle for two-site DMRG (test infrastructure only).

This package exists to check the GPU library.  Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the library and its Python binding
never do.  It shares no code with the CUDA path.

Contents (each function cites the passage of the block2 paper, arXiv 2310.03920, it
follows):
  ops          local Fock basis and elementary operators (Listing 1, Part A)
  hamiltonian  ab initio Hamiltonian as a list of site-ordered operator strings (Sec. 2.1.1)
  fci          determinant full CI, first-quantised two-electron check, Hubbard-Holstein FCI
  mpo          exact MPO from the operator strings: a prefix tree (the general MPO
               construction of Sec. 2.3)
  dmrg         environments, effective Hamiltonian, Davidson, truncation and the two-site
               sweep (Sec. 2.1.2)
  rdm          one- and two-particle density matrices (Sec. 2.5.1)
"""
