"""FP64 CPU oracle — test infrastructure only (tests, smoke check, CPU baseline)."""

from .oracle import *  # noqa: F401,F403
from .oracle import lib, num_threads  # noqa: F401
