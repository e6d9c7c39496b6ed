"""GB300-native non-Fourier SENSE reconstruction: E, E^H and CG on sm_103a kernels."""
