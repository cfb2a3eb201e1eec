"""GB300-native lattice Boltzmann step for self-diffusiophoretic particles near
and at liquid-liquid interfaces (arXiv 2202.01631).

Submodules:
  lbdp       ctypes binding of the CUDA C-ABI library liblbdp.so
  build      in-tree build of liblbdp.so for sm_103a
  workloads  seeded synthetic inputs
"""
__all__ = ["lbdp", "build", "workloads"]
