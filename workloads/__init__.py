"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the
benchmark.  Nothing here computes any step of the refinement method."""
