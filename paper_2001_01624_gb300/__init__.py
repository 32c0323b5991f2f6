"""GB300-native multiscale multibasis pressure solver.

Hot path (hand-written CUDA for sm_103a behind the C ABI in include/ms.h):
two-point flux assembly, MsRSB prolongation bases with partition-of-unity
renormalisation, dynamically adapted extra bases from pressure updates,
Galerkin coarse operators with dense coarse factorisation, and the
multiscale multibasis Richardson solve with an ILU(0) or Jacobi smoother.

``binding`` exposes the C entry points under their own names; ``geomodel``
builds seeded synthetic inputs; ``build`` compiles the library in-tree.
"""
from . import geomodel  # noqa: F401
from .binding import *  # noqa: F401,F403
from .binding import MsError, lib  # noqa: F401
