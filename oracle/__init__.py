"""CPU FP64 oracle -- test infrastructure only (see td_oracle.py)."""
from .td_oracle import *  # noqa: F401,F403
from .td_oracle import NotPositiveDefinite, OracleSegment  # noqa: F401
