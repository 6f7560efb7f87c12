"""GB300-native Video Complexity Analyzer hot path (C-ABI library libvca.so + ctypes binding).

The seven per-frame features of Section 2 of the paper (E_Y, h, L_Y, E_U, E_V, L_U, L_V)
are computed by hand-written sm_103a CUDA kernels behind the C ABI in include/vca.h.
Import ``paper_2304_12384_gb300.vca`` for the binding; ``build.build()`` compiles the
library in-tree.
"""

__all__ = ["build", "vca"]
