"""GB300-native FMM for screened-Coulomb (linearized Poisson-Boltzmann) potentials and fields
of charges in layered media (Wang, Zhang & Cai, arXiv 2002.01334).

The compute path is the C-ABI library ``liblpbfmm.so`` (hand-written sm_103a CUDA kernels);
``paper_2002_01334_gb300.lpbfmm`` is a thin ctypes binding with the same entry points.
``paper_2002_01334_gb300.inputs`` generates seeded synthetic workloads;
``paper_2002_01334_gb300.multigpu`` splits one evaluation across GPUs (one process each).
"""
__all__ = ["lpbfmm", "inputs", "multigpu"]
