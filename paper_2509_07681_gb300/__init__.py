"""GB300-native FUnc-SNE: the per-iteration step as hand-written CUDA
behind a C ABI (``include/funcsne.h``), with a thin Python binding.

Import ``paper_2509_07681_gb300.funcsne`` for the binding; this package
initialiser stays import-light so that ``synth`` and ``quality`` load
without the CUDA library.
"""
__all__ = ["funcsne", "synth", "quality"]
