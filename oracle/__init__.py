"""CPU FP64 oracle (test infrastructure only; never imported by the GPU library)."""
from .rpa_oracle import *  # noqa: F401,F403
