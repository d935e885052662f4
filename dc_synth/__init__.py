"""Seeded synthetic diffusion-curve drawings.

This module is shared by the oracle (tests only) and by the GPU path's tests
and benchmark.  It draws random numbers and rejects bad samples; it holds
none of the boundary-integral method's arithmetic.  Geometry here is a dense
polyline sampling of each Bezier curve, used only to decide acceptance
(simplicity, separation) and how many times a panel is bisected.  Every
value it returns is an exact input of the method: control points, colours,
and panel break points given as dyadic fractions of each curve's arc length.

Workloads stand in for the paper's drawings (Orzan 2008 and others, which
are not available): curve counts and shapes follow the sizes quoted in the
paper's timing tables (32 to 4632 curves on a unit canvas).
"""
from .drawings import (  # noqa: F401
    Drawing,
    make_closed_set,
    make_mixed_set,
    drawing_by_name,
    random_node_values,
    pixel_sample,
    viewport_set,
    curve_point,
    circle_loops,
    curve_tangent,
)
from . import harmonic  # noqa: F401
