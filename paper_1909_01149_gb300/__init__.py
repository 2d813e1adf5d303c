"""GB300-native alternating-update NNCP (PLANC, arXiv 1909.01149).

The compute path lives in the C-ABI library ``libplanc.so`` (hand-written
sm_103a CUDA under ``csrc/``); ``planc`` is its thin ctypes binding.  The
binding is imported lazily so that ``synth`` (seeded inputs) can be used on a
machine without the built library.
"""

import importlib

__all__ = ["planc", "synth"]


def __getattr__(name):
    if name in ("planc", "synth"):
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
