"""FP64 CPU oracle of the FUnc-SNE iteration (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package. It shares no code with the CUDA path.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import __all__  # noqa: F401
