"""Seeded synthetic inputs: circuits, their wire cuts and the subcircuit
variant outputs (the QPU stand-in).  Shared by the oracle tests and the CUDA
path; holds none of the reconstruction arithmetic."""
