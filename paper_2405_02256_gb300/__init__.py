"""GB300-native topological integral transforms (critical tables, ECT, Radon, hybrid).

The compute path is the CUDA library ``libtopot.so`` (C ABI declared in
``include/topot.h``); ``binding`` is a thin ctypes layer over it.  Importing the
package does not load the library; the first call that needs it does, and raises if
it is missing -- there is no CPU fallback.
"""
__all__ = ["synth", "binding"]
