"""GB300-native DG operator of arXiv:1805.01443 (placeholder, binding added below)."""
