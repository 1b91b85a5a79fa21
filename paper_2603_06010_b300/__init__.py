"""B300-native time-domain Gaussian likelihood (arXiv 2603.06010 hot path).

Importing the package loads nothing native; `td.lib()` loads the C-ABI
library (libtd.so) and raises if it is missing.
"""
__all__ = ["inputs", "td"]
