"""FP64 CPU oracle for the IFDLBM step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. The
product path (the CUDA library and its Python binding) never imports it and
shares no code with it.
"""
from .ifdlbm import *  # noqa: F401,F403
