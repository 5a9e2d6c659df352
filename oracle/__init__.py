"""Plain FP64 CPU oracle for the extinction-mapping hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the tests, the package's smoke check and the benchmark's CPU-baseline
leg may call it.  It shares no code with the CUDA library.
"""
from .gmead_oracle import *  # noqa: F401,F403
