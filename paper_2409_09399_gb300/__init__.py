"""GB300-native real-space grid integration (gint) for numerical-atomic-orbital DFT.

The compute path is libgint.so (hand-written CUDA for sm_103a behind the C ABI
in include/gint.h); ``gint.Gint`` is its Python binding.
"""
from .gint import Gint, GintError, from_system, load, PRECISIONS  # noqa: F401
from .autograd import GintEnergy, energy, energy_and_strain  # noqa: F401
