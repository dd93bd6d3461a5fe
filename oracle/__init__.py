"""Plain FP64 CPU oracle for messenger mapmaking: test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline legs may
import this package.  It shares no code with the CUDA path.
"""
from .messenger import *  # noqa: F401,F403
