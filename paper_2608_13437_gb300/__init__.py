"""GB300 library for the fused time step of the compressible Navier-Stokes-Fourier
lattice Boltzmann scheme (Bukreev, Kummerlaender, Krause).

Modules:
  lbm     -- ctypes binding of liblbm.so (the C ABI in include/lbm.h)
  build   -- in-tree nvcc build of liblbm.so for sm_103a
  inputs  -- seeded synthetic workloads (TGV, Sod, batched TGV domains)
"""
__all__ = ["lbm", "build", "inputs"]
