"""Compressed-frontier BFS for GB300 (sm_103a)."""
