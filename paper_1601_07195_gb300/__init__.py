"""GB300 state-vector gate engine: the data-parallel core of qHiPSTER
(arXiv:1601.07195) as hand-written sm_103a CUDA behind a C ABI (include/qs.h).

``qs`` is the ctypes binding; ``build`` compiles libqs.so in-tree.
"""

from . import qs  # noqa: F401
from .qs import State, Plan, QSError, grad  # noqa: F401
