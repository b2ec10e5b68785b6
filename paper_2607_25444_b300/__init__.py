"""B300-native (sm_103a) conservative Allen-Cahn lattice Boltzmann wetting
step (arXiv 2607.25444).

- ``csrc/``: the CUDA kernels and the C ABI declared in ``include/cacl.h``.
- ``cacl``: the Python binding of ``libcacl.so`` (marshalling only).
- ``inputs``: seeded synthetic inputs (geometries, droplets, parameters).
- ``build``: compiles ``libcacl.so`` in-tree for sm_103a.
"""
