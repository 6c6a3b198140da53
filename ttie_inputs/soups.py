"""Seeded triangle soups for pair-level tests.

A soup is a set of triangles that share no vertices, so every i<j pair is
non-adjacent.  ``snapped_soup`` puts vertices on a coarse integer grid so that
degenerate configurations (vertex on a plane, shared planes, touching
intervals, coplanar pairs) occur often.
"""
from __future__ import annotations

import numpy as np

from .meshes import Mesh


def triangle_soup(n_tri: int, seed: int, box: float = 1.0, size: float = 0.6) -> Mesh:
    """n_tri random triangles: a random centre in [0, box]^3 plus three offsets in
    [-size, size]^3, so neighbouring triangles overlap often."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.0, box, (n_tri, 1, 3))
    x = (c + rng.uniform(-size, size, (n_tri, 3, 3))).reshape(-1, 3)
    tri = np.arange(3 * n_tri, dtype=np.int32).reshape(n_tri, 3)
    return Mesh(x, tri, np.zeros(n_tri, np.int32))


def snapped_soup(n_tri: int, seed: int, grid: int = 3) -> Mesh:
    """Triangles with integer vertex coordinates in [0, grid]^3 (non-degenerate triangles only).

    Small grids make exact degeneracies common: coplanar pairs, a vertex lying on the
    other triangle's plane, collinear edges, touching intervals."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n_tri:
        t = rng.integers(0, grid + 1, (3, 3)).astype(np.float64)
        if np.linalg.norm(np.cross(t[1] - t[0], t[2] - t[0])) > 0:
            out.append(t)
    x = np.concatenate(out)
    tri = np.arange(3 * n_tri, dtype=np.int32).reshape(n_tri, 3)
    return Mesh(x, tri, np.zeros(n_tri, np.int32))


def closed_form_pair(alpha0: float, alpha1: float, beta0: float, beta1: float, h: float = 0.7) -> Mesh:
    """Two triangles whose plane-cut segments lie on the x axis.

    Triangle A lies in z=0 with vertices (0,-h,0), (2*alpha0,h,0), (2*alpha1,h,0); the plane
    y=0 cuts it in the x-interval [alpha0, alpha1].  Triangle B lies in y=0 with vertices
    (0,0,-h), (2*beta0,0,h), (2*beta1,0,h); the plane z=0 cuts it in [beta0, beta1]."""
    x = np.array([[0.0, -h, 0.0], [2 * alpha0, h, 0.0], [2 * alpha1, h, 0.0],
                  [0.0, 0.0, -h], [2 * beta0, 0.0, h], [2 * beta1, 0.0, h]])
    tri = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    return Mesh(x, tri, np.array([0, 1], np.int32))
