"""FP64 CPU oracle (test infrastructure only; see nsp_oracle for the rules)."""
from .nsp_oracle import *  # noqa: F401,F403
from . import nsp_oracle  # noqa: F401
