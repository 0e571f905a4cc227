"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds meshes (node coordinates and element-to-node connectivity),
seeded random draws (circle parameters, stream-function coefficients) and the
workload descriptions (which mesh, order, velocity field and initial interface).
It holds none of the flux-reconstruction arithmetic: no solution points, no
operators, no fluxes. Both the CPU oracle and the CUDA path consume what it
produces and each evaluates the method on its own.
"""
from .meshes import (Mesh, quad_grid, tri_delaunay, tri_split, hex_grid)
from .workloads import (Velocity, Circle, SlottedDisk, Workload, workload, WORKLOADS,
                        stream_coefficients, ensemble_instances, initial_phi)

__all__ = ["Mesh", "quad_grid", "tri_delaunay", "tri_split", "hex_grid",
           "Velocity", "Circle", "SlottedDisk", "Workload", "workload", "WORKLOADS",
           "stream_coefficients", "ensemble_instances", "initial_phi"]
