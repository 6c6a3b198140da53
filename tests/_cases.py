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


# Required agreement with the FP64 oracle, on pairs whose min(|t_c^0|, |t_c^1|) exceeds
# MASK_REL times the bounding-box diagonal: T relative 1e-5, gradients and Hessian blocks
# relative 1e-4 (gradient and Hessian norm-wise per pair: largest entry error over largest
# entry).  The same numbers hold for the FP32 and the FP64 form.
T_RTOL = 1e-5
G_RTOL = 1e-4
H_RTOL = 1e-4
MASK_REL = 1e-6


def tolerance_mask(x, tc_oracle):
    """Pairs the stated tolerances apply to: min(|t_c^0|, |t_c^1|) > MASK_REL * diagonal."""
    diag = float(np.linalg.norm(np.asarray(x).max(0) - np.asarray(x).min(0)))
    return np.minimum(np.abs(tc_oracle[:, 0]), np.abs(tc_oracle[:, 1])) > MASK_REL * diag


def pair_errors(tc, dtc, ev, psd="per_part"):
    """Per-pair relative errors of the GPU's t_c and t_c gradients (rows matching the oracle's
    PairEval ev, all intersecting) against the oracle: T, the Eq. 3 gradient and the projected
    Eq. 4 Hessian (the oracle's projection applied to the GPU's values), each as the largest
    entry error over the largest oracle entry.  Returns (eT, eg, eH)."""
    import oracle as O
    tc = np.asarray(tc, np.float64)
    dtc = np.asarray(dtc, np.float64).reshape(-1, 2, 18)
    T_gpu = (tc[:, 0] * tc[:, 1]) ** 2
    eT = np.abs(T_gpu - ev.T) / np.abs(ev.T)
    evg = O.PairEval(ev.pairs, tc, dtc, ev.sides64, ev.flags64, ev.active)
    g_gpu, g_or = O.gradient(evg), O.gradient(ev)
    eg = np.abs(g_gpu - g_or).max(1) / np.abs(g_or).max(1)
    H_gpu, H_or = O.hessian_psd(evg, psd), O.hessian_psd(ev, psd)
    n = len(tc)
    eH = np.abs(H_gpu - H_or).reshape(n, -1).max(1) / np.abs(H_or).reshape(n, -1).max(1)
    return eT, eg, eH


def block_errors(got, blocks):
    """Assembled 3x3 blocks {(row vertex, col vertex): block} against the oracle's: the
    Frobenius error of each block over sqrt(|H_rr| |H_cc|) (the scale that bounds an
    off-diagonal block of a PSD matrix).  Returns the array of those ratios."""
    dn = {k[0]: np.linalg.norm(b) for k, b in blocks.items() if k[0] == k[1]}
    return np.array([np.linalg.norm(got[k] - b) / np.sqrt(dn[k[0]] * dn[k[1]]) for k, b in blocks.items()])
