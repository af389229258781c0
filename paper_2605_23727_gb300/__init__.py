"""GB300 (sm_103a) mixed-precision Bogacki-Shampine 3(2) solver for large,
densely coupled ODE systems.

The compute path is the CUDA library ``libbs3.so`` (C ABI in include/bs3.h);
``bs3`` is its ctypes binding.  Importing this package does not load the
library; ``bs3.load()`` does, and raises if it has not been built.
"""

from . import bs3  # noqa: F401

__all__ = ["bs3"]
