"""GB300 (sm_103a) Chebyshev random-probe tight-binding path of arXiv 1812.05264.

``api`` holds the torch-facing calls (neighbour list, H assembly, spectral bounds, moments,
chemical potential, density matrix and forces, an end-to-end ``Solver`` and the ``FreeEnergy``
autograd function); ``_lib`` is the ctypes binding of ``libtbk.so`` (include/tbk.h); ``build``
compiles the library in-tree.  Importing the package does not load CUDA code.
"""
