"""Seeded synthetic inputs for the spatio-temporal BTA workloads.

This package produces *inputs only*: mesh geometry (node coordinates and
triangles), observation sites (location, containing triangle, time step,
response variable), covariates, observed values and the generating
hyperparameter vector.  It holds none of the method's arithmetic: no finite
element matrices, no interpolation weights, no precision matrices.  Both the
CPU oracle (``oracle/``) and the CUDA path (``paper_2507_06938_gb300``) read
these arrays and build everything else themselves.
"""

from .generate import (  # noqa: F401
    Problem,
    CONFIGS,
    grid_mesh,
    delaunay_mesh,
    make_problem,
    problem_from_config,
    theta_layout,
)
