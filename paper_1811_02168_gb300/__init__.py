"""GB300-native Fourier bilateral filtering (Optimized Fourier Bilateral Filtering, IEEE SPL 2018).

Import is light: ``synth`` (input generator) needs no native code.  The binding loads
``libfbf.so`` on first use and raises if it is missing -- there is no CPU fallback.
"""
__all__ = ["binding", "synth", "build"]


def __getattr__(name):
    if name in ("binding", "synth", "build"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
