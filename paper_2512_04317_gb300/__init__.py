"""GB300-native MX-scaled low-precision 2D FFT (arXiv 2512.04317)."""
