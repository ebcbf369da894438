"""GB300-native two-phase sparse matrix-matrix multiply (C = A·B on CSR).

The method is the paper's kkSpGEMM (Deveci, Trott, Rajamanickam): a symbolic
phase on a column-set-compressed B computes C's row pointers, a numeric phase
accumulates C's rows with Gustavson's algorithm into multi-level hash or dense
accumulators.  All computation runs in ``libkkspgemm.so`` (hand-written CUDA for
sm_103a) behind the C ABI of ``include/kkspgemm.h``; this package only
marshals arguments.
"""

from ._binding import SpGEMMError, load as load_library  # noqa: F401

__all__ = ["SpGEMMError", "load_library", "ops"]
__version__ = "0.1.0"


def __getattr__(name):
    if name == "ops":
        import importlib
        return importlib.import_module(__name__ + ".ops")
    raise AttributeError(name)
