"""GB300-native monodomain reaction-diffusion step (BeatBox, arXiv:1605.06015).

The compute path is the CUDA library ``libbbx.so`` built from ``csrc/`` and
reached through the C ABI declared in ``include/bbx.h``; ``bbx`` is its thin
ctypes binding.  ``workloads`` holds the seeded synthetic input generators.
Importing the package loads nothing; ``from paper_1605_06015_gb300 import bbx``
loads the library and fails loudly if it has not been built.
"""
__all__ = ["bbx", "workloads"]
