"""GB300-native DVBM time step (double-distribution quasi-equilibrium model)."""
