"""pgc -- GB300-native speculative graph coloring (D1, D2, PD2)."""
