"""GB300-native semi-implicit Fourier pseudo-spectral phase-field-crystal step."""
