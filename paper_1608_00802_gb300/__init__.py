"""GB300-native particle-mesh step with quantum pressure (arXiv:1608.00802)."""
