"""Hardware probes used to place kernels on their roofline (not part of the library)."""
