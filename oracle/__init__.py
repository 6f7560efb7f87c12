"""CPU oracle for the Video Complexity Analyzer hot path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs
of ``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or calls it.
"""

from .vca_oracle import *  # noqa: F401,F403
