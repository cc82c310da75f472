"""B300-native HEALPix spherical Gaussian rasterizer (UniTriSplat, arXiv 2606.29794)."""
