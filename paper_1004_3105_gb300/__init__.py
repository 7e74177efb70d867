"""GB300-native normal variate generators (Brent's Algorithms B1 and P)."""
