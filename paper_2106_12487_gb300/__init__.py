"""GB300-native FFT-based Bloch-wave dispersion (Segurado & Lebensohn, arXiv 2106.12487)."""
