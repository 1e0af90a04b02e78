"""GB300-native fast Slepian projection (arXiv:1611.04950).

The binding lives in ``paper_1611_04950_gb300.fst`` (C names of include/fst.h plus
the ``Plan`` wrapper); its names are re-exported here on first use, so that the
build script and the workload generators import without the compiled library.
Importing the binding without libfst_gb300.so raises ImportError.
"""
import importlib as _importlib


def __getattr__(name):
    if name.startswith("__") or name in ("fst", "build", "workloads"):
        raise AttributeError(name)
    return getattr(_importlib.import_module(__name__ + ".fst"), name)
