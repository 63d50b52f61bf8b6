"""GB300-native SL1M hot path (Hardy 2013): matrix-free forward operator,
adjoint and positivity-constrained FISTA as sm_103a CUDA kernels behind the
C ABI of ``libsl1m``.  The binding lives in :mod:`paper_1310_2078_gb300.sl1m`
(imported lazily so that the input generator can be used without the
compiled library)."""

__all__ = ["sl1m", "synth"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
