"""GB300-native piCholesky cross-validation (arXiv 1404.0466).

The compute path lives in ``libpichol.so`` (hand-written sm_103a CUDA behind a
C ABI, declared in ``include/pichol.h``); ``binding`` marshals arguments to it,
``autotune`` times its launch-shape choices, and ``synth`` draws seeded
synthetic workloads.  Importing the package does not load the library;
``binding.lib()`` does, and raises if it has not been built.
"""
__all__ = ["autotune", "binding", "synth"]
