"""Seeded synthetic triangle meshes for the TTIE workloads.

This module holds geometry generation only: vertex positions, triangle index
rows and per-triangle group ids.  It contains none of the intersection-energy
arithmetic, so both the CUDA path and the CPU oracle may draw their inputs from
it.  Every generator is deterministic for a given seed
(``numpy.random.default_rng``).

Returned meshes are ``Mesh(x, tri, group)``:
  x     float64 [V, 3]  vertex positions
  tri   int32   [F, 3]  vertex indices, counter-clockwise seen from outside
  group int32   [F]     mesh / instance id of each triangle
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Mesh:
    x: np.ndarray
    tri: np.ndarray
    group: np.ndarray

    @property
    def V(self) -> int:
        return int(self.x.shape[0])

    @property
    def F(self) -> int:
        return int(self.tri.shape[0])

    def as_f32(self) -> "Mesh":
        """Positions rounded to float32 and returned as float64 (exact copy of the f32 values)."""
        return Mesh(self.x.astype(np.float32).astype(np.float64), self.tri, self.group)


def concat(meshes) -> Mesh:
    xs, tris, groups = [], [], []
    off = 0
    for g, m in enumerate(meshes):
        xs.append(m.x)
        tris.append(m.tri + off)
        groups.append(np.full(m.F, g, np.int32))
        off += m.V
    return Mesh(np.concatenate(xs), np.concatenate(tris).astype(np.int32),
                np.concatenate(groups).astype(np.int32))


# ---------------------------------------------------------------- rotations
def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation from a normalised Gaussian quaternion."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def rot_x(deg: float) -> np.ndarray:
    c, s = np.cos(np.radians(deg)), np.sin(np.radians(deg))
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]], dtype=np.float64)


# ---------------------------------------------------------------- subdivision
def _midpoint_subdivide(x: np.ndarray, tri: np.ndarray):
    """Split every triangle into four; shared edge midpoints are deduplicated."""
    F = tri.shape[0]
    e = np.stack([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]], axis=1).reshape(-1, 2)
    e_sorted = np.sort(e, axis=1)
    uniq, inv = np.unique(e_sorted, axis=0, return_inverse=True)
    inv = inv.reshape(F, 3)
    mid = 0.5 * (x[uniq[:, 0]] + x[uniq[:, 1]])
    m = inv + x.shape[0]
    a, b, c = tri[:, 0], tri[:, 1], tri[:, 2]
    mab, mbc, mca = m[:, 0], m[:, 1], m[:, 2]
    new_tri = np.concatenate([
        np.stack([a, mab, mca], 1),
        np.stack([b, mbc, mab], 1),
        np.stack([c, mca, mbc], 1),
        np.stack([mab, mbc, mca], 1),
    ])
    return np.concatenate([x, mid]), new_tri.astype(np.int32)


def icosphere(subdiv: int = 2, radius: float = 1.0) -> Mesh:
    """Icosahedron (golden-ratio vertices) subdivided ``subdiv`` times, projected to the sphere.

    subdiv=2 gives V=162, F=320.
    """
    p = (1.0 + 5.0 ** 0.5) / 2.0
    x = np.array([[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
                  [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
                  [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]], dtype=np.float64)
    tri = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                    [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                    [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                    [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int32)
    for _ in range(subdiv):
        x, tri = _midpoint_subdivide(x, tri)
    x = radius * x / np.linalg.norm(x, axis=1, keepdims=True)
    return Mesh(x, tri, np.zeros(tri.shape[0], np.int32))


def octasphere(level: int, radius: float = 1.0) -> Mesh:
    """Octahedron subdivided ``level`` times, projected to the sphere: F = 8*4**level."""
    x = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], np.float64)
    tri = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4],
                    [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]], np.int32)
    for _ in range(level):
        x, tri = _midpoint_subdivide(x, tri)
    x = radius * x / np.linalg.norm(x, axis=1, keepdims=True)
    return Mesh(x, tri, np.zeros(tri.shape[0], np.int32))


def edge_list(tri: np.ndarray) -> np.ndarray:
    """[E,2] int32 undirected edges (i < j) of a triangle mesh, each once, sorted (topology for
    the springs of the quasi-static simulation's workloads)."""
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]]).astype(np.int64)
    e.sort(axis=1)
    return np.unique(e, axis=0).astype(np.int32)


# ---------------------------------------------------------------- grids
def grid_sheet(n: int):
    """n x n vertex grid on [0,1]^2, every quad split along the same diagonal: F = 2(n-1)^2."""
    u = np.linspace(0.0, 1.0, n)
    X, Y = np.meshgrid(u, u, indexing="xy")
    idx = np.arange(n * n, dtype=np.int32).reshape(n, n)
    a = idx[:-1, :-1].ravel()
    b = idx[:-1, 1:].ravel()
    c = idx[1:, 1:].ravel()
    d = idx[1:, :-1].ravel()
    tri = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)]).astype(np.int32)
    return X.ravel(), Y.ravel(), tri


def sinusoid_field(rng, n_terms=8, amp=(0.05, 0.3), wavenumber=(2.0, 12.0)):
    """Draw a seeded sum of plane-wave sinusoids; returns f(x, y)."""
    A = rng.uniform(*amp, n_terms)
    w = rng.uniform(*wavenumber, n_terms)
    th = rng.uniform(0, 2 * np.pi, n_terms)
    ph = rng.uniform(0, 2 * np.pi, n_terms)

    def f(x, y):
        out = np.zeros_like(x)
        for k in range(n_terms):
            out += A[k] * np.sin(2 * np.pi * w[k] * (x * np.cos(th[k]) + y * np.sin(th[k])) + ph[k])
        return out
    return f


def cloth(n: int = 256, seed: int = 2, crossing: bool = True, shear: float = 0.4) -> Mesh:
    """Self-intersecting cloth sheet.

    z = sum of 8 seeded sinusoids (amplitude U[0.05,0.3], wavenumber U[2,12] cycles/unit).
    ``crossing=False``: x <- x + shear*z, which is a linear bijection of a height field and
    therefore leaves the sheet intersection-free.  ``crossing=True`` (default): x <- x +
    shear*g(x, y) with g an independent second 8-sinusoid field, which folds the sheet
    through itself along curves.
    """
    rng = np.random.default_rng(seed)
    X, Y, tri = grid_sheet(n)
    fz = sinusoid_field(rng)
    Z = fz(X, Y)
    if crossing:
        g = sinusoid_field(rng)
        Xs = X + shear * g(X, Y)
    else:
        Xs = X + shear * Z
    x = np.stack([Xs, Y, Z], 1)
    return Mesh(x, tri, np.zeros(tri.shape[0], np.int32))


def torus(R: float = 1.0, r: float = 0.3, n_major: int = 256, n_minor: int = 128) -> Mesh:
    i = np.arange(n_major)
    j = np.arange(n_minor)
    I, J = np.meshgrid(i, j, indexing="ij")
    u = 2 * np.pi * I / n_major
    v = 2 * np.pi * J / n_minor
    x = np.stack([(R + r * np.cos(v)) * np.cos(u), (R + r * np.cos(v)) * np.sin(u), r * np.sin(v)], -1)
    x = x.reshape(-1, 3)
    idx = (I * n_minor + J)
    a = idx
    b = ((I + 1) % n_major) * n_minor + J
    c = ((I + 1) % n_major) * n_minor + (J + 1) % n_minor
    d = I * n_minor + (J + 1) % n_minor
    a, b, c, d = a.ravel(), b.ravel(), c.ravel(), d.ravel()
    tri = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)]).astype(np.int32)
    return Mesh(x, tri, np.zeros(tri.shape[0], np.int32))


def ellipsoid(n_lat: int, semi_axes) -> Mesh:
    """Latitude-longitude ellipsoid with n_lon = 2 n_lat: F = 2 n_lon (n_lat - 1)."""
    n_lon = 2 * n_lat
    th = np.pi * np.arange(1, n_lat) / n_lat
    ph = 2 * np.pi * np.arange(n_lon) / n_lon
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    ring = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    x = np.concatenate([[[0, 0, 1]], ring, [[0, 0, -1]]]) * np.asarray(semi_axes)[None, :]
    top, bot = 0, 1 + (n_lat - 1) * n_lon
    tris = []
    k = np.arange(n_lon)
    r0 = 1 + k
    tris.append(np.stack([np.full(n_lon, top), r0, 1 + (k + 1) % n_lon], 1))
    for ring_i in range(n_lat - 2):
        base0 = 1 + ring_i * n_lon
        base1 = base0 + n_lon
        a = base0 + k
        b = base1 + k
        c = base1 + (k + 1) % n_lon
        d = base0 + (k + 1) % n_lon
        tris.append(np.stack([a, b, c], 1))
        tris.append(np.stack([a, c, d], 1))
    base = 1 + (n_lat - 2) * n_lon
    tris.append(np.stack([base + k, np.full(n_lon, bot), base + (k + 1) % n_lon], 1))
    tri = np.concatenate(tris).astype(np.int32)
    return Mesh(x, tri, np.zeros(tri.shape[0], np.int32))


# ---------------------------------------------------------------- value noise
class ValueNoise3:
    """Seeded lattice value noise: random values at integer lattice points, smoothstep-weighted
    trilinear interpolation, ``octaves`` octaves (lacunarity 2, gain 0.5), range [-1, 1]."""

    def __init__(self, rng, base_freq=8.0, octaves=5, table=256):
        self.base_freq = base_freq
        self.octaves = octaves
        self.table = table
        self.perm = [rng.permutation(table) for _ in range(octaves)]
        self.vals = [rng.uniform(-1, 1, table) for _ in range(octaves)]

    def _lattice(self, o, i, j, k):
        p = self.perm[o]
        n = self.table
        return self.vals[o][p[(p[(p[i % n] + j) % n] + k) % n]]

    def __call__(self, pts: np.ndarray) -> np.ndarray:
        out = np.zeros(pts.shape[0])
        amp, freq, norm = 1.0, self.base_freq, 0.0
        for o in range(self.octaves):
            q = pts * freq
            f = np.floor(q)
            t = q - f
            s = t * t * (3 - 2 * t)
            i0 = f.astype(np.int64)
            acc = np.zeros(pts.shape[0])
            for dx in (0, 1):
                wx = s[:, 0] if dx else 1 - s[:, 0]
                for dy in (0, 1):
                    wy = s[:, 1] if dy else 1 - s[:, 1]
                    for dz in (0, 1):
                        wz = s[:, 2] if dz else 1 - s[:, 2]
                        acc += wx * wy * wz * self._lattice(o, i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz)
            out += amp * acc
            norm += amp
            amp *= 0.5
            freq *= 2.0
        return out / norm


# ---------------------------------------------------------------- workloads
def two_icospheres(seed: int = 1, offset=(1.2, 0.0, 0.0)) -> Mesh:
    """Two radius-1 icospheres (320 triangles each); the second is randomly rotated and moved
    to ``offset`` so the surfaces interpenetrate.  group = 0 / 1 per sphere."""
    rng = np.random.default_rng(seed)
    a = icosphere(2)
    b = icosphere(2)
    Rm = random_rotation(rng)
    b = Mesh(b.x @ Rm.T + np.asarray(offset)[None, :], b.tri, b.group)
    return concat([a, b])


def interlocked_tori(seed: int = 3, offset=(0.5, 0.0, 0.0), n_major=256, n_minor=128,
                     jitter=0.005) -> Mesh:
    """Two tori (R=1, r=0.3); the second rotated 90 degrees about x and moved by ``offset``,
    plus seeded Gaussian vertex jitter.  ``offset=(1,0,0)`` keeps the tubes apart;
    ``offset=(0.5,0,0)`` makes them interpenetrate."""
    rng = np.random.default_rng(seed)
    a = torus(1.0, 0.3, n_major, n_minor)
    b = torus(1.0, 0.3, n_major, n_minor)
    b = Mesh(b.x @ rot_x(90.0).T + np.asarray(offset)[None, :], b.tri, b.group)
    m = concat([a, b])
    m.x = m.x + rng.normal(0.0, jitter, m.x.shape)
    return m


def noisy_sphere(level: int = 9, seed: int = 5, amplitude: float = 0.15, vector: bool = True) -> Mesh:
    """Octahedral sphere (F = 8*4**level) displaced by 5-octave value noise (base frequency 8).

    ``vector=False``: radial displacement amplitude*N(p) along the normal (a radial graph,
    hence intersection-free).  ``vector=True`` (default): displacement amplitude*(N1,N2,N3)(p)
    by three independent noise fields, which folds the surface through itself."""
    rng = np.random.default_rng(seed)
    m = octasphere(level)
    p = m.x
    if vector:
        disp = np.stack([ValueNoise3(rng)(p) for _ in range(3)], 1)
        x = p + amplitude * disp
    else:
        x = p * (1.0 + amplitude * ValueNoise3(rng)(p))[:, None]
    return Mesh(x, m.tri, m.group)


def ellipsoid_batch(n_instances: int = 512, seed: int = 4, f_min=100, f_max=20000):
    """Batch of independent ellipsoid pairs with log-uniform triangle counts.

    Returns (mesh, vertex_offsets, tri_offsets); group[f] = instance id, and each instance's
    two ellipsoids are placed with a random relative rotation and a centre offset of
    U[0.3, 1.0] x (mean semi-axis of A + mean semi-axis of B) along a random direction."""
    rng = np.random.default_rng(seed)
    parts = []
    for inst in range(n_instances):
        pair = []
        for _ in range(2):
            target = np.exp(rng.uniform(np.log(f_min), np.log(f_max)))
            n_lat = max(3, int(round((1 + np.sqrt(1 + target)) / 2)))
            # F = 4 n_lat (n_lat - 1); choose the n_lat nearest to the target
            cands = [n_lat - 1, n_lat, n_lat + 1]
            n_lat = min((c for c in cands if c >= 3), key=lambda c: abs(4 * c * (c - 1) - target))
            axes = rng.uniform(0.5, 1.5, 3)
            pair.append((ellipsoid(n_lat, axes), axes))
        (ma, axa), (mb, axb) = pair
        Rm = random_rotation(rng)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        off = d * rng.uniform(0.3, 1.0) * (axa.mean() + axb.mean())
        mb = Mesh(mb.x @ Rm.T + off[None, :], mb.tri, mb.group)
        inst_mesh = concat([ma, mb])
        inst_mesh.group[:] = inst
        parts.append(inst_mesh)
    vo = np.cumsum([0] + [p.V for p in parts]).astype(np.int64)
    to = np.cumsum([0] + [p.F for p in parts]).astype(np.int64)
    m = concat(parts)
    m.group = np.concatenate([p.group for p in parts]).astype(np.int32)
    return m, vo, to
