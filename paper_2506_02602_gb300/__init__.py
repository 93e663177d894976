"""GB300-native per-cell chemistry integrator (low-storage RK, Eq. 21-22).

``chem`` is the Python binding of libchem.so (include/chem.h); ``build`` compiles it
in-tree for sm_103a.
"""
from . import build, chem  # noqa: F401
