"""B300-native (sm_103a) double-distribution lattice Boltzmann library with
consistent body force and heat source for compressible flows of generic
fluids (arxiv 2609.28679).  The compute path is the CUDA library liblbm.so
(C ABI in include/lbm.h); ``lbm`` is its Python binding and ``workloads``
holds the seeded synthetic inputs."""

__all__ = ["lbm", "workloads", "build"]
