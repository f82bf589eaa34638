"""Plain FP64 CPU oracle of the D3Q27 MRT lattice Boltzmann step (test infrastructure).

This package is TEST INFRASTRUCTURE.  It computes, slowly and literally, what the
paper (arXiv 2405.12082, Sec. II.A, Sec. II.B, Sec. II.C and Appendix A) defines:
the 27x27 moment transform, the printed equilibrium and forcing moments, the MRT
relaxation, two-buffer pull streaming with bounce-back, the trigger force and the
coherent-structure mode analysis.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  The CUDA library never
imports, links or calls anything here, and nothing here imports the CUDA library.

Modules
  lattice    velocity set, weights, moment matrix M^T and its exact inverse
  collision  Hermite equilibrium, printed m_eq and R, the MRT collision
  lbm        geometry, forces, streaming, initial state, time loop, statistics
  modes      ring sampling, R_uu correlation, its DFT power and the dominant mode
  rng        SplitMix64 counter-based generator and Box-Muller normals
  adjoint    reverse-mode of the step (dual-number collision Jacobian)
"""
