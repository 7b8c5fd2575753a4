"""GB300-native spectral split-step Pade (SSSP) parabolic-equation range marcher."""
