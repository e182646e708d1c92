"""GB300-native real-space FLO-SIC orbital-SIC step (arxiv 2108.01186)."""
