"""FP64 CPU oracle: test infrastructure only (see shs_oracle's header)."""
from .shs_oracle import *  # noqa: F401,F403
from .shs_oracle import Config, shade_forward, shade_backward  # noqa: F401
