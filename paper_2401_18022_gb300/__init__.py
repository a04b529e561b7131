"""GB300-native ISRS GN integral model (arXiv 2401.18022)."""
