"""GB300 hot path of SIMP topology optimisation on dynamically refined octree
meshes (Wang, de Sturler, Paulino): a C-ABI CUDA library (libtm.so, see
include/tm.h) and its Python binding ``paper_1009_4975_gb300.tm``."""
from . import tm  # noqa: F401
from .tm import *  # noqa: F401,F403
