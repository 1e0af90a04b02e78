"""FP64 CPU oracle for the fast Slepian projection.  Test infrastructure only:
imported by the tests, the smoke check and the benchmark's CPU-baseline leg,
never by the library."""
from .fst_oracle import *  # noqa: F401,F403
