"""GB300-native hierarchization of sparse-grid combination grids (placeholder;
the CUDA library binding lands next)."""
