"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the
benchmark.  Holds random draws and input assembly only: none of the
rasterizer's arithmetic lives here."""
