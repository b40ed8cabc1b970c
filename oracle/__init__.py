"""CPU oracle for the shifted Green's-function solve.

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct FP64
implementations of what the GPU library computes, written from the method
(Eq. 1, Eq. 2, Sec. 3, Sec. 8) and sharing no code with the library.  Only
tests/, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg may
import, call, link or execute anything under oracle/.

Modules:
  philox      Philox4x32-10 and the uniform/normal conversions
  systems     lattices, neighbour lists, BSR H and S
  dense       exact G by dense LU and by eigen-decomposition; closed forms
  cocg        plain FP64 shifted COCG on CSR (C, OpenMP over columns)
  gf          LDOS and density-matrix reductions of G
  subspace    hop-shell local subspaces and principal submatrices
  mlp         FP64 multilayer perceptron forward/backward and Adam
  descriptors per-column local-environment descriptors
"""
