"""GB300-native engine for the Mapple index-mapping hot path (arxiv 2507.17087)."""
