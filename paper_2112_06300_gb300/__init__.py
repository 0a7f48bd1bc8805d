"""GB300-native continuous collision detection (sweep-and-prune broad phase
and conservative interval-bisection narrow phase)."""
