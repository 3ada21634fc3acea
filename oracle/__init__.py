"""FP64 CPU oracle (test infrastructure only; never used by the product path).

See ``oracle.cs_oracle`` for the functions and the passages they follow.
"""
from .cs_oracle import *  # noqa: F401,F403
