"""GB300 phase-field lattice Boltzmann step (arXiv 2512.01032).

The compute path is the CUDA library ``_lib/libpflb.so`` behind the C ABI of
``include/pflb.h``; ``pflb`` is its ctypes binding.  There is no CPU
fallback: calls fail when the library or a CUDA device is missing.
"""
from . import pflb  # noqa: F401
from .pflb import Lattice, PflbError, default_params, load  # noqa: F401
