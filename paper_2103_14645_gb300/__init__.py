"""GB300-native renderer for baked Sparse Neural Radiance Grids (SNeRG, arXiv 2103.14645)."""
