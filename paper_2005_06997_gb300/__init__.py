"""GB300-native nonlocal hydrodynamic FDTD (arXiv 2005.06997)."""
