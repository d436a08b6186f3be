"""GB300-native short-range nonbonded forces (LJ + Ewald real-space Coulomb).

The compute path is libnb.so (CUDA for sm_103a, C ABI in include/nb.h);
``nb`` is its Python binding and ``engine`` the rolling-prune driver.
"""
from . import nb  # noqa: F401
from .nb import Pairlist, NBError  # noqa: F401
