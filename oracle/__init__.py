"""FP64 CPU oracle (test infrastructure only; see lpf_oracle)."""
from .lpf_oracle import *  # noqa: F401,F403
from . import lpf_oracle  # noqa: F401
