"""Worker for process pools that run the FP64 oracle beside a GPU test.  The pool must use
the spawn start method: the parent already holds a CUDA context.  Imports only numpy and
the oracle.  Each worker keeps its BLAS and OpenMP libraries to one thread (the workers
already cover the cores; nested thread pools oversubscribe them badly)."""
import os

for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

from oracle import fst_oracle as O  # noqa: E402


def oracle_fast(args):
    """(N, W, eps, y) -> the oracle's fast projection of y with its own plan (K = round(2NW))."""
    N, W, e, y = args
    return O.fast_project(O.make_plan(N, W, O.default_K(N, W), e), np.asarray(y, dtype=np.float64))
