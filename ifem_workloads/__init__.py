"""Seeded synthetic inputs (meshes, particle placements, MAC velocity fields).

Shared by the CPU oracle tests and the CUDA path; holds none of the
coupling-step arithmetic.
"""
from .configs import Box, Instance, Template, Workload, make  # noqa: F401
