"""GB300-native particle SMC over PPL control-flow graphs (PCFGs).

The compute path is the CUDA library ``libsmc.so`` (sources in ``csrc/``,
C ABI in ``include/smc.h``); ``smc`` is its ctypes binding.
"""
from . import smc  # noqa: F401

__all__ = ["smc"]
