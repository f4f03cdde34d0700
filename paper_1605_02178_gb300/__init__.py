"""GB300-native Gauss-Chebyshev bilateral filter (Ghosh & Chaudhury 2016).

The compute path is the C-ABI library libbfgc.so (include/bfgc.h) built from
csrc/ for sm_103a; ``bfgc`` binds it with the same names and ``api`` adds a plan
object and an autograd Function.  Importing this package does not load the
library; the first call does, and raises if it cannot.
"""
__all__ = ["bfgc", "api", "synth"]
