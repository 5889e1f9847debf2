"""GB300-native Fast Selective Extrapolation (Seiler & Kaup, arXiv 2204.14194)."""
