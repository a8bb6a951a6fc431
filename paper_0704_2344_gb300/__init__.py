"""GB300-native nodal finite-element H-field scattering solver.

Submodules (imported on demand, nothing is loaded eagerly):
  fe         - ctypes binding of the C ABI in include/fe.h (libfe_gb300.so)
  build      - compiles csrc/*.cu for sm_103a into libfe_gb300.so
  workloads  - seeded synthetic voxel problems and plane-wave sets
"""
