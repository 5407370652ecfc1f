"""GB300-native FFT-correlator system for redundant arrays on a regular grid
(Gorthi, Parsons & Dillon 2020).

Submodules:
  gridcorr -- binding of the C ABI in include/gridcorr.h (loads libgridcorr.so)
  synth    -- seeded synthetic voltages (input generator only)
  _build   -- in-tree nvcc build of libgridcorr.so

The binding is imported lazily so that the input generator works on hosts
where the CUDA library has not been built; any call into the hot path goes
through `gridcorr`, which raises if the library is missing.
"""
import importlib

__all__ = ["gridcorr", "synth"]


def __getattr__(name):
    if name in ("gridcorr", "synth", "_build"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
