"""GB300-native soft-decision Viterbi decoder (arxiv 2011.09337).

The decoder lives in the CUDA library ``libvit.so`` built from ``csrc/``; the
Python side (:mod:`.vit`) only marshals torch tensors through its C ABI.  The
library is loaded on first use and a missing build raises immediately: there
is no CPU fallback.
"""
from importlib import import_module

__all__ = ["vit", "synth"]


def __getattr__(name):
    if name in ("vit", "synth", "tune"):
        return import_module(f".{name}", __name__)
    raise AttributeError(name)
