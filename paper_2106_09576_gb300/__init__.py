"""GB300-native hot path of the soft-sphere DEM method of Lethe-DEM (arXiv 2106.09576).

The compute path is libdem_gb300.so (CUDA, sm_103a) behind the C ABI in include/dem.h;
``dem.DEM`` is its Python binding.  ``build.build()`` compiles the library in-tree.
"""
from . import build
from .dem import DEM, DemError, load_library

__all__ = ["DEM", "DemError", "load_library", "build"]
