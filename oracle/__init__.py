"""FP64 CPU oracle for the plane-wave Hamiltonian hot path.

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, plain, independent
statement of what the GPU library computes.  Only ``tests/``, the smoke check
in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import,
call, link or execute anything in this directory.  It shares no code with the
CUDA library and never imports it.

Modules:
  cfft        plain C transforms (direct DFT, recursive Cooley-Tukey, direct 3-D)
  planewave   basis, local potential, projectors, operators I J Idag Jdag O,
              apply_H, density, subspace, dense Hamiltonian
  minimize    band conjugate-gradient minimiser (Teter / MLP / identity)
  mlp         the FP64 reference of the per-coefficient preconditioner network
  scf         Hartree potential, LDA exchange-correlation, Pulay mixing and the
              self-consistent field loop around dense band solves
  pcm         the linear dielectric Poisson solve (hessian, CG, A_diel)
  spinor      two-component bands in a noncollinear potential: H C, n and m
  ultrasoft   augmented overlap S = Omega + P Q P^dag and generalised Rayleigh-Ritz
"""
