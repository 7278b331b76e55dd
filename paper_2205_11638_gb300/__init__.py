"""GB300 (sm_103a) BDD Lagrange-dual solver: the data-parallel hot path of
DOGE-Train (arXiv 2205.11638) behind the C ABI of ``include/dg.h``.

``solver`` is the thin PyTorch binding (argument marshalling only),
``build`` compiles ``csrc/`` into ``_build/libdg.so``.
"""
from .solver import (Arena, DualIterate, Graph, LowerBound, NonParamUpdate, ParamTransform, Plan,  # noqa: F401
                     make_options, plan)
