"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This package holds none of the method's arithmetic: it draws random numbers,
evaluates phantom coefficient fields xi(x) on a grid and lists the workload
shapes.  Forward modelling (turning xi into data W) is done by the oracle on the
CPU or by the library's own forward kernel on the GPU, never here.
"""
from .phantoms import (gaussian_inclusions, random_gaussians, sphere_phantom,
                       noise_direction, grid_points, three_bumps)
from .workloads import PaperWorkload, Workload, WORKLOADS, paper_workload, workload

__all__ = ["gaussian_inclusions", "random_gaussians", "sphere_phantom",
           "noise_direction", "grid_points", "three_bumps", "PaperWorkload", "Workload", "WORKLOADS",
           "paper_workload", "workload"]
