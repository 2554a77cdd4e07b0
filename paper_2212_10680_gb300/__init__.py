"""GB300-native (sm_103a) fugacity-based multicomponent lattice Boltzmann.

The compute path is libfmlbm.so (CUDA C++, C ABI in include/fmlbm.h); ``fmlbm`` is
its ctypes binding (imported on demand, it fails loudly when the library is not
built); ``inputs`` builds seeded synthetic initial fields; ``build`` compiles the
library in-tree with nvcc for sm_103a.
"""
__all__ = ["fmlbm", "inputs", "build"]
__version__ = "0.1.0"
