"""GB300-native application of sequences of planar rotations (placeholder; binding added with the library)."""
