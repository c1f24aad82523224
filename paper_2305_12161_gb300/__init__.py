"""GB300-native zero-temperature checkerboard quench of the d=3 Ising model (arXiv:2305.12161)."""
