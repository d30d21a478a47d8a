"""Seeded synthetic inputs for cone-beam backprojection.

This package only *generates* inputs: scan geometries (one 3x4 projection
matrix per view, plus the source/detector description they were built from),
volume grids, and analytic projections of an ellipsoid phantom with FDK-style
cosine weighting and Shepp-Logan ramp filtering.  It contains none of the
backprojection arithmetic.  Both the CUDA path and the FP64 oracle consume
what it produces; neither is imported here.

The workloads stand in for the RabbitCT rabbit dataset (496 C-arm
projections of 1248x960 FP32 pixels, one 3x4 matrix per view, a 512^3
volume; Section "RabbitCT Benchmark" of the paper), which is not available.
"""
from .geometry import ScanGeometry, short_scan, volume_grid, orthographic_matrix
from .phantom import Phantom, random_phantom, project_phantom, ramp_filter_rows, make_projections
from .workloads import Workload, make_workload, WORKLOADS

__all__ = [
    "ScanGeometry", "short_scan", "volume_grid", "orthographic_matrix",
    "Phantom", "random_phantom", "project_phantom", "ramp_filter_rows", "make_projections",
    "Workload", "make_workload", "WORKLOADS",
]
