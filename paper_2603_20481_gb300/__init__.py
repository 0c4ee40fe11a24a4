"""GB300-native RISE: complex IQ captures -> spectrogram -> detected energy boxes.

The compute path is the CUDA library built from `csrc/` (C ABI in
`include/rise.h`); `rise` is its Python binding and `synth` the seeded
synthetic-capture generator used by the tests and the bench.
"""
from . import synth  # noqa: F401  (input generator only)

__all__ = ["synth", "rise", "build"]


def __getattr__(name):
    if name in ("rise", "build"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
