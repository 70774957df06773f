"""GB300 (sm_103a) Geant4-style navigation and gamma transport.

The compute path lives in ``libg4nav.so`` (hand-written CUDA behind a C ABI,
declared in ``include/g4nav.h``); this package is its thin Python binding
(argument marshalling only).  PyTorch supplies device memory and streams.
"""
from .binding import *  # noqa: F401,F403
from .binding import __all__  # noqa: F401
