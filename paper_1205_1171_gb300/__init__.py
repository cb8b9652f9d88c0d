"""GB300-native kinetic divide-and-conquer 3D convex hull (White & Wortman, Sec. 2-3)."""
