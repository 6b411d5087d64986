"""GB300 (sm_103a) s-step GMRES with two-stage block orthogonalization.

The compute path is the CUDA library ``libgmres.so`` built from ``csrc/``
(see ``build.py``) behind the C ABI declared in ``include/gmres.h``;
``capi`` is its thin ctypes binding.  Importing this package does not load
the library; ``capi.load()`` does, and fails loudly when it is missing.
"""
__all__ = ["capi", "build"]
