"""Seeded synthetic inputs shared by the CUDA path's tests and the CPU oracle.

Geometry only: no step of the intersection-energy method lives here.
"""
from .meshes import (Mesh, concat, edge_list, icosphere, octasphere, cloth, torus, ellipsoid,  # noqa: F401
                     two_icospheres, interlocked_tori, noisy_sphere, ellipsoid_batch,
                     random_rotation, grid_sheet)
from .soups import triangle_soup, closed_form_pair, snapped_soup  # noqa: F401
