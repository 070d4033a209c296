"""FP64 CPU oracle of the SPOD hot path -- test infrastructure only.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline / reference legs may import this package.  It shares no code with the
CUDA library and never imports it.
"""
from .spod_oracle import *  # noqa: F401,F403
from . import spod_oracle  # noqa: F401
