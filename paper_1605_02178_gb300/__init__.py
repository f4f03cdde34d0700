"""GB300-native Gauss-Chebyshev bilateral filter (Ghosh & Chaudhury 2016)."""
