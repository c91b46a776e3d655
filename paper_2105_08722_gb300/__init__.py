"""GB300-native implementation of the ENCORE isotropic NPCF estimator (arXiv:2105.08722).

The estimator runs in ``libencore_gpu.so`` (CUDA, sm_103a); this package holds the
ctypes binding (``NPCF``), the build step and the seeded synthetic catalogs.
"""
from .build import build  # noqa: F401


def __getattr__(name):
    if name in ("NPCF", "NPCFError", "FP32", "SPLIT_BF16", "load"):
        from . import _lib
        return getattr(_lib, name)
    raise AttributeError(name)
