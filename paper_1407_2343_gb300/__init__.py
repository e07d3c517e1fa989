"""GB300-native separable non-local means (Ghosh & Chaudhury, arXiv:1407.2343).

The computation lives in libsnlm.so (hand-written sm_103a CUDA behind a C ABI,
include/snlm.h); ``api`` is its Python binding with the same entry-point names.
Submodules are imported lazily so that ``synth`` (the input generator) can be
used without the CUDA library.
"""

__all__ = ["api", "synth", "build"]


def __getattr__(name):
    import importlib

    if name in ("api", "synth", "build", "batch", "serve", "autotune"):
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
