"""GB300-native push-relabel additive approximation for OT (arXiv 2203.03732)."""
