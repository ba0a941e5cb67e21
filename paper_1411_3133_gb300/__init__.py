"""GB300-native lattice Boltzmann for generalized metrics.

Hot path: the fused collide-and-stream update of the lattice Boltzmann model
in curvilinear coordinates (Debus, Mendoza, Herrmann, "Dean Instability in
Double-Curved Channels", Sec. II-IV) as hand-written sm_103a CUDA kernels
behind the C ABI of include/lbgm.h (liblbgm.so).

Modules
  build      compile liblbgm.so in-tree with nvcc (sm_103a)
  lbgm       ctypes binding of the C ABI (same function names)
  workloads  seeded synthetic channel workloads (no method arithmetic)
"""
