"""CPU oracle for the Viola-Jones AdaBoost round (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package.  The library path never does.
"""

from .oracle import *  # noqa: F401,F403
