"""FP64 CPU oracle (test infrastructure only; see randutv_oracle)."""
from .randutv_oracle import *  # noqa: F401,F403
