"""B300-native batched quantum-trajectory TEBD for the Lindblad equation.

The compute path is the CUDA library liblindtebd.so (C ABI in include/lindtebd.h);
`lindtebd` is its ctypes binding.  Importing the package raises ImportError when
the library has not been built: there is no CPU fallback.
"""
from . import lindtebd  # noqa: F401
from .lindtebd import Ensemble, LtError  # noqa: F401
