"""GB300-native EAPrunedDTW subsequence search (placeholder, filled in below)."""
