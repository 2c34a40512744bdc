"""GB300-native pseudopotential MRT lattice Boltzmann step (arXiv:1605.01800).

- ``include/lbm.h`` + ``csrc/``: the C-ABI CUDA library ``liblbm.so`` (sm_103a).
- ``lbm``: the Python binding of that ABI (same function names).
- ``inputs``: seeded synthetic workloads shaped like the paper's cases.
- ``build``: in-tree nvcc build of ``liblbm.so``.
"""
