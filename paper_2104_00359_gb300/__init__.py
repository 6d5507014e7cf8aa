"""GB300-native SH soft-shadow shading (Lyu et al., arXiv 2104.00359).

The hot path -- per-point SH visibility from a sphere set, the clamped-cosine
lobe, the SH triple product and the lighting contraction, forward and
adjoint -- runs in hand-written sm_103a CUDA kernels behind the C ABI in
include/shs.h.  ``shade`` / ``Scene`` are the PyTorch-facing entry points.
"""

from .shade import Config, Scene, ShadeFunction, shade  # noqa: F401
