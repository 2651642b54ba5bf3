"""Windowed regularized LBM-LES and its discrete adjoint on one B300 (sm_103a).

Submodules:
  binding   ctypes binding of liblbmadj.so (the C ABI of include/lbmadj.h)
  autograd  torch.autograd.Function mapping the design field to J_eff
  inputs    seeded synthetic problem inputs
  build     nvcc build of the in-tree library

Importing the package loads nothing; the CUDA library is loaded on first use
and its absence raises.
"""
