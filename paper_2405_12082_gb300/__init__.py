"""GB300-native D3Q27 MRT pipe-flow lattice Boltzmann library (arXiv 2405.12082).

The compute path is the CUDA library built from csrc/ (C ABI in include/lbm.h);
``paper_2405_12082_gb300.lbm`` is its ctypes binding and
``paper_2405_12082_gb300.workloads`` the seeded synthetic workloads.  Submodules
are imported on demand so that the workload definitions load without the library.
"""
__all__ = ["lbm", "workloads", "build"]
