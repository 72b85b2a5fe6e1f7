"""Seeded synthetic inputs for the cut-cell Poisson method (arXiv:1411.4283).

This package is an INPUT GENERATOR shared by the FP64 oracle (``oracle/``) and
the GPU library (``paper_1411_4283_gb300``).  It holds none of the
discretisation's arithmetic: it builds analytic geometries (circles in 2D,
spheres in 3D), integrates functions over the cut cells, grid faces and
embedded-boundary (EB) patches of a Cartesian grid (``geom.c``; ellipses in
``ellipse.py``), and draws the
seeded random numbers the workloads need (SplitMix64).

The moment tables it produces are the inputs the paper takes from its
geometry generator (Sec. 2.1, volume / face / normal-weighted moments; Sec. 3.1
asks for O(h^{6+D}) accurate moments).  Here they are exact to rounding.
"""
from .geometry import (Geometry, monomials, circle_config, four_circles_config, multi_circle_config, multi_sphere_config,
                       sphere_box_config, sphere_inside_config, line_config, ProductFn, level_set_modes)
from .ellipse import EllipseGeometry, ellipse_batch_config
from .rng import SplitMix64, uniform, seeded_field
from .manufactured import Manufactured, sin_product

__all__ = ["Geometry", "monomials", "circle_config", "four_circles_config", "multi_circle_config", "multi_sphere_config",
           "sphere_box_config", "sphere_inside_config", "line_config", "ProductFn", "level_set_modes", "SplitMix64", "uniform",
           "seeded_field", "Manufactured", "sin_product", "EllipseGeometry", "ellipse_batch_config"]
