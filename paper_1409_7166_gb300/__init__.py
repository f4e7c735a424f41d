"""GB300-native topology-based transient analysis of power grids.

The CUDA library (``_lib/libpg.so``, sources in ``csrc/``, C ABI in
``include/pg.h``) does the work; :mod:`.binding` marshals arguments to it.
Importing this package does not load the library; ``binding.lib()`` does and
raises if it is missing.
"""
from .build import build, LIB  # noqa: F401
