"""B300-native matrix-free high-order Lagrangian hydrodynamics hot path.

The compute path lives in the C-ABI shared library `liblh.so` (CUDA kernels
for sm_103a, see `csrc/`); `paper_2112_07075_b300.lh` is its thin ctypes
binding. `paper_2112_07075_b300.inputs` generates seeded synthetic meshes.
Importing this package loads nothing; the binding loads the library on first use.
"""
