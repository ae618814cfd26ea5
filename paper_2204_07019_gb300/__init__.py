"""GB300-native micro-continuum dissolution step (Maes, Soulaine & Menke,
"Improved Volume-of-Solid formulations for micro-continuum simulation of
mineral dissolution at the pore-scale").

The compute path is the CUDA library ``libvos.so`` (built from ``csrc/``)
behind the C ABI declared in ``include/vos.h``; :mod:`.vos` is the thin
ctypes binding.  :mod:`.inputs` holds the seeded geometry / parameter
generators and is importable without a GPU or the compiled library.
"""

__all__ = ["inputs", "vos"]


def __getattr__(name):
    # Lazy: importing the package must not load the CUDA library.
    if name in ("vos", "inputs"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
