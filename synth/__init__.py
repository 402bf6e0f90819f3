"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This package generates meshes (node coordinates, element connectivity,
boundary-face tags, periodic translations, and for curved meshes each
element's quadratic node coordinates, placed on the straight element and
moved by a smooth map, as a mesh generator would) and closed-form initial
conditions evaluated at caller-supplied coordinates, and seeded initial
network weights.  It holds none of the
flux-reconstruction arithmetic: no solution/flux points, no operators, no
geometry factors, no face matching.  Both implementations compute those on
their own from what this package returns.
"""
from .meshgen import (  # noqa: F401
    BC_WALL, BC_FARFIELD, ETYPE_TET, ETYPE_PRI, ETYPE_HEX, TET_FACES, PRI_FACES, HEX_FACES,
    layered_box, vortex_box, hex_box, boundary_layer_box, wall_channel, tgv_box, batch_problem_params,
    batch_problem_mesh, mesh_counts, curve_mesh, QUAD_NODES,
)
from .ics import (  # noqa: F401
    isentropic_vortex, taylor_green, perturbed_freestream, uniform_state,
    random_smooth_state, shear_flow, shear_wave,
)
from .weights import mlp_init  # noqa: F401
