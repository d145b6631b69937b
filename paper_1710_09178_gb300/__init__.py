"""GB300-native even-odd staggered multi-shift CG (placeholder, filled in below)."""
