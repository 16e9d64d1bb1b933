"""GB300-native time step of the generalized lattice Boltzmann model for flow
through tight porous media with Klinkenberg's effect (Chen et al.,
arXiv:1411.7051).

* ``lbmp``   -- Python binding of the C ABI (``include/lbmp.h``) of the CUDA
  library ``_lib/liblbmp.so`` (sm_103a kernels in ``csrc/``).
* ``media``  -- seeded synthetic porous media (inputs only).
* ``build``  -- in-tree nvcc build of the library.
"""
