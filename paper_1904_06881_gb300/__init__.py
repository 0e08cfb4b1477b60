"""GB300-native ternary high-density-ratio free-energy lattice Boltzmann step
with wetting boundaries (arXiv:1904.06881)."""
