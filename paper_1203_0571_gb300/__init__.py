"""libfse: GB300-native fast shape estimation for galaxies and stars.

Li, Xin & Cui (2012): weighted-moment centroid, KSB ellipticity with an
elliptical weight, and a Sérsic profile fit over (r_e, n) with the amplitude
at its closed form, over many postage stamps at once.  The computation lives
in hand-written sm_103a CUDA kernels behind the C ABI of include/fse.h; this
package is its ctypes binding (``binding``) plus a seeded stamp generator
(``synth``) for tests and benchmarks.
"""
from __future__ import annotations

__all__ = ["binding", "synth"]


def __getattr__(name):
    # the binding is imported lazily so that `synth` needs no CUDA toolkit
    import importlib
    if name in ("binding", "synth"):
        return importlib.import_module(f"{__name__}.{name}")
    if name in ("Context", "default_opts", "make_index", "results"):
        return getattr(importlib.import_module(f"{__name__}.binding"), name)
    raise AttributeError(name)
