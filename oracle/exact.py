"""Exact rational form of the paper's intersection test (oracle; test infrastructure only).

The test of §1 (Eq. 1 and the open criterion 0 in (t_c^0, t_c^1)) evaluated in
``fractions.Fraction`` arithmetic on the exact binary values of the inputs.
Two positive scalings are dropped because they change no sign and no
comparison: the normalisation of the cutting-plane normal (the crossing
points are ratios of the d_k) and the normalisation of the line direction D
(t = D.(S - O) becomes w.S with w = n_B x n_A, which only rescales and shifts
every t by the same amounts).  Zero tests are exact, so the census follows
§1's case analysis with the degenerate cases decided exactly (a vertex on the
plane counts as zero; touching intervals do not overlap).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def _sub(a, b):
    return (a[0] - b[0], a[1] - b[1], a[2] - b[2])


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def _sign(v):
    return (v > 0) - (v < 0)


def _crossing(qm, dm, qp, dp):
    """Point where the edge (qm, qp) meets the plane: (dp qm - dm qp) / (dp - dm)."""
    den = dp - dm
    return tuple((dp * qm[k] - dm * qp[k]) / den for k in range(3))


def plane_cut(P, Q):
    """Cut triangle Q by the plane of triangle P.

    Returns (segment or None, signs): the segment when Q straddles the plane
    (some vertex strictly on each side), and the exact side of each Q_k."""
    n = _cross(_sub(P[1], P[0]), _sub(P[2], P[0]))
    d = [_dot(n, _sub(Q[k], P[k])) for k in range(3)]
    s = [_sign(v) for v in d]
    pos, neg = s.count(1), s.count(-1)
    if not (pos > 0 and neg > 0):
        return None, s
    if pos + neg == 2:
        z = s.index(0)
        p, q = sorted([(z + 1) % 3, (z + 2) % 3])
        return (Q[z], _crossing(Q[p], d[p], Q[q], d[q])), s
    lone = 1 if pos == 1 else -1
    m = s.index(lone)
    p, q = sorted([(m + 1) % 3, (m + 2) % 3])
    return (_crossing(Q[m], d[m], Q[p], d[p]), _crossing(Q[m], d[m], Q[q], d[q])), s


def _frac_tri(x, t):
    return [tuple(Fraction(float(c)) for c in x[v]) for v in t]


def pair_active_exact(A, B) -> bool:
    """Exact value of the paper's test for triangles A, B given as 3 Fraction 3-tuples."""
    segB, _ = plane_cut(A, B)
    if segB is None:
        return False
    segA, _ = plane_cut(B, A)
    if segA is None:
        return False
    nA = _cross(_sub(A[1], A[0]), _sub(A[2], A[0]))
    nB = _cross(_sub(B[1], B[0]), _sub(B[2], B[0]))
    w = _cross(nB, nA)
    tA = [_dot(w, s) for s in segA]
    tB = [_dot(w, s) for s in segB]
    return max(tA) > min(tB) and min(tA) < max(tB)


def pair_sides_exact(A, B):
    """Exact sides [B_k vs plane A (3), A_k vs plane B (3)]."""
    _, sB = plane_cut(A, B)
    _, sA = plane_cut(B, A)
    return sB + sA


def active_exact(x: np.ndarray, tri: np.ndarray, pairs: np.ndarray, prefilter=None) -> np.ndarray:
    """Exact active flag of every pair (rows of ``pairs`` index ``tri``).

    ``prefilter`` (optional, [P, 6] int8 from the certified FP64 side filter) lets
    pairs whose census is certainly one-sided in either direction skip the rational
    evaluation; it never decides a pair that might be active."""
    out = np.zeros(len(pairs), dtype=bool)
    cache = {}

    def tri_of(f):
        t = cache.get(f)
        if t is None:
            t = _frac_tri(x, tri[f])
            cache[f] = t
        return t

    for p, (i, j) in enumerate(pairs):
        if prefilter is not None:
            s = prefilter[p]
            if (np.all(s[:3] == 1) or np.all(s[:3] == -1) or
                    np.all(s[3:] == 1) or np.all(s[3:] == -1)):
                continue
        out[p] = pair_active_exact(tri_of(int(i)), tri_of(int(j)))
    return out
