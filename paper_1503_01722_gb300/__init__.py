"""GB300-native coupled photon-electron Monte Carlo dose engine (method of
Tian et al., oclMC). The compute path is the CUDA library libocmc.so behind the
C ABI in include/ocmc.h; ``paper_1503_01722_gb300.ocmc`` is its thin ctypes
binding. There is no CPU fallback: loading fails loudly without the library.
"""
__version__ = "0.1.0"


def __getattr__(name):
    if name in ("ocmc",):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
