"""GB300 (sm_103a) lattice Boltzmann stream-and-collide library (arXiv 2305.09910).

``lbm`` is the ctypes binding of the C ABI (include/lbm.h) implemented by ``liblbm.so``;
``inputs`` holds the seeded synthetic input generators; ``build`` compiles the library.
Submodules are imported on demand so that importing the package does not load CUDA.
"""
__all__ = ["lbm", "inputs", "build"]
