"""GB300-native cost tables for MesonGS++'s size-aware configuration search.

The compute path is libmgs.so (CUDA, sm_103a) behind include/mgs.h; `mgs` is
its ctypes binding, `synth` draws seeded synthetic scenes, `build` compiles
the library in-tree.
"""
from . import synth  # noqa: F401

__all__ = ["mgs", "synth", "build"]
