"""GB300-native FNR impulse filter for infrared frames (arXiv 1201.3972).

The compute path is the C-ABI library built from ``csrc/``; this package is
its thin Python binding. Importing the package does not load the library;
the first call that needs it does, and raises if it is missing.
"""
__all__ = ["synth"]
