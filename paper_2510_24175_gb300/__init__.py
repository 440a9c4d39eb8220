"""GB300-native GLM-MHD hot path (placeholder; binding added below)."""
