"""Seeded test workloads and comparison helpers shared by the GPU tests."""
import numpy as np

import ttie_inputs as ti


def small_cases():
    """name -> (mesh with float32-representable positions, pair mode name).

    Sizes span several 32-pair warps, 2048-key sort tiles and a ragged tail."""
    return {
        "cloth40": (ti.cloth(40, seed=2, shear=0.3).as_f32(), "self"),
        "cloth_literal33": (ti.cloth(33, seed=2, crossing=False).as_f32(), "self"),
        "spheres_inter": (ti.two_icospheres().as_f32(), "inter"),
        "soup": (ti.triangle_soup(700, seed=12, size=0.35).as_f32(), "self"),
        "snapped_grid": (ti.snapped_soup(260, seed=13, grid=3).as_f32(), "self"),
        "tori": (ti.interlocked_tori(offset=(0.5, 0, 0), n_major=40, n_minor=20).as_f32(), "self"),
        "ellipsoids_intra": (_ellipsoids(), "instance"),
    }


def _ellipsoids():
    m, _, _ = ti.ellipsoid_batch(6, seed=4, f_min=60, f_max=600)
    return m.as_f32()


MODE = {"self": 0, "inter": 1, "instance": 2}


def pair_set(p):
    p = np.asarray(p, dtype=np.int64).reshape(-1, 2)
    return set(map(tuple, p.tolist()))


def fp32_tolerance(T, g, L, kappa=64.0):
    """Tolerance of an FP32 evaluation against the FP64 value: relative 1e-5 plus the change of T
    under a position perturbation of kappa * u32 * L (u32 = 2^-24, L = size of the pair)."""
    return 1e-5 * np.abs(T) + kappa * 2.0 ** -24 * L * np.abs(g).sum(axis=-1)
