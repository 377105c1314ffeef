"""GB300 (sm_103a) population likelihood of "Parallelized Inference for
Gravitational-Wave Astronomy" (Sec. "Population acceleration").

``binding`` is the ctypes binding of libpop.so (C-ABI in include/pop.h);
``synth`` draws seeded synthetic catalogs and injections; ``build`` compiles the
CUDA library in-tree.
"""
from . import binding, synth  # noqa: F401
from .binding import Likelihood  # noqa: F401

__all__ = ["binding", "synth", "Likelihood"]
