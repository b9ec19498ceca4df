"""GB300-native variational multiscale Newton-Schur assembly for 3D incompressible Navier-Stokes.

Submodules:
  inputs  - seeded synthetic meshes, Dirichlet sets and flow states (no method arithmetic)
  vms     - thin ctypes binding of the C-ABI library libvms_gb300.so (loaded on first use)
  build   - nvcc build of the CUDA library for sm_103a
"""
__all__ = ["inputs", "vms", "build"]
