"""FP64 CPU oracle of the TTIE hot path (test infrastructure only).

Every function restates one step of "Differentiable 3D Triangle-Triangle
Intersection Energy" plainly, in FP64, so a reader can check it against the
paper.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline use it; the CUDA path never imports it.

Steps and the passages they follow:
  candidate_pairs   all i<j pairs sharing no vertex (§1: topologically adjacent
                    pairs are excluded), optionally restricted to closed AABB
                    overlap; brute force O(F^2).
  evaluate          per pair: t_c^0, t_c^1 and their gradients (Appendix A,
                    forward-mode duals, ``pair_dual.c``); exact active flag
                    (``exact.py``); T (Eq. 2), gradient (Eq. 3), inexact
                    Hessian (Eq. 4), eigen-analysis projection (§1.1).
  assemble          sum of per-pair 18-vectors / 18x18 blocks over vertices.
  hessian_vector_product  exact Hessian of T (no Eq. 4 terms dropped) times a
                    direction: derivative of the Eq. 3 gradient along it,
                    fourth-order central differences at fixed pairs, the
                    step refined per pair until it lies in one smooth piece.
  newton_solve      inexact Newton with backtracking line search until no pair
                    intersects (abstract, §1.2 "GPU-based inexact Newton").

Readings where the paper is silent or at odds with itself:
  * t_c scale: Eq. 1 has t_c^0 = t_a^0 - t_b^1; the appendix returns half of
    it.  ``tc_scale`` = 1 (Eq. 1) by default, 0.5 reproduces the appendix.
  * T = (t_c^0 t_c^1)^2 only on intersecting pairs, 0 otherwise (Eq. 2 applies
    to intersecting pairs; the open criterion of §1 decides which those are).
  * The active decision is exact (rational arithmetic), not the FP64
    comparison of the listing.
  * Eigen-analysis (§1.1): parts 1 and 2 of Eq. 4 are PSD; part 3 is projected
    by clamping its negative eigenvalues to zero (per-part projection).
  * Newton details (regularisation, tolerances, line search) are not given;
    the policy is stated in ``NewtonParams``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

from . import exact

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libttie_oracle.so")
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile pair_dual.c (plain C, FP64, no FMA contraction) into oracle/_build."""
    src = os.path.join(_HERE, "pair_dual.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        P = ctypes.c_void_p
        lib.ttie_oracle_eval.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_double, P, P, P, P]
        lib.ttie_oracle_sides.argtypes = [P, P, P, ctypes.c_int64, P]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ pairs
def adjacent(tri: np.ndarray, i, j) -> np.ndarray:
    """True where triangles i and j share at least one vertex index (§1: adjacent)."""
    ti, tj = tri[i], tri[j]
    return (ti[:, :, None] == tj[:, None, :]).any(axis=(1, 2))


def tri_aabb(x: np.ndarray, tri: np.ndarray):
    v = x[tri]                      # F x 3 x 3
    return v.min(axis=1), v.max(axis=1)


def candidate_pairs(x: np.ndarray, tri: np.ndarray, group=None, mode: str = "self",
                    aabb: bool = True, chunk: int = 2048) -> np.ndarray:
    """All i<j pairs (int64 [P,2], lexicographic order) that share no vertex, filtered by mode:
    'self' all pairs, 'inter' only group[i] != group[j], 'instance' only group[i] == group[j];
    with ``aabb`` only pairs whose closed bounding boxes overlap."""
    F = tri.shape[0]
    lo, hi = tri_aabb(x, tri)
    out = []
    for s in range(0, F, chunk):
        e = min(F, s + chunk)
        ii = np.arange(s, e)
        m = np.arange(F)[None, :] > ii[:, None]
        if aabb:
            m &= np.all(lo[ii][:, None, :] <= hi[None, :, :], axis=2)
            m &= np.all(lo[None, :, :] <= hi[ii][:, None, :], axis=2)
        if group is not None and mode == "inter":
            m &= group[ii][:, None] != group[None, :]
        elif group is not None and mode == "instance":
            m &= group[ii][:, None] == group[None, :]
        a, b = np.nonzero(m)
        a = a + s
        keep = ~adjacent(tri, a, b)
        out.append(np.stack([a[keep], b[keep]], 1))
    return np.concatenate(out).astype(np.int64) if out else np.zeros((0, 2), np.int64)


def partners_of(x, tri, i: int, group=None, mode="self") -> np.ndarray:
    """Sorted j (any order relation to i, j != i) whose closed AABB overlaps that of i and that
    share no vertex with i, under the pair mode: the brute-force candidate row of triangle i."""
    lo, hi = tri_aabb(x, tri)
    m = np.all(lo[i][None, :] <= hi, axis=1) & np.all(lo <= hi[i][None, :], axis=1)
    m[i] = False
    if group is not None and mode == "inter":
        m &= group != group[i]
    elif group is not None and mode == "instance":
        m &= group == group[i]
    j = np.nonzero(m)[0]
    j = j[~adjacent(tri, np.full(len(j), i), j)]
    return j


# ------------------------------------------------------------------ per pair
@dataclass
class PairEval:
    pairs: np.ndarray      # [P,2] triangle ids (i, j)
    tc: np.ndarray         # [P,2] t_c^0, t_c^1 (Eq. 1, times tc_scale)
    dtc: np.ndarray        # [P,2,18] gradients of t_c^0, t_c^1 w.r.t. [A0 A1 A2 B0 B1 B2]
    sides64: np.ndarray    # [P,6] FP64 census signs
    flags64: np.ndarray    # [P] bit0 B straddles A, bit1 A straddles B, bit2 FP64 overlap
    active: np.ndarray     # [P] exact active flag

    @property
    def T(self):
        """Eq. 2: T = (t_c^0 t_c^1)^2 on intersecting pairs."""
        return np.where(self.active, (self.tc[:, 0] * self.tc[:, 1]) ** 2, 0.0)


def eval_pairs_f64(x: np.ndarray, tri: np.ndarray, pairs: np.ndarray, tc_scale: float = 1.0):
    """FP64 forward-mode evaluation of every pair (no active decision)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    pairs = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
    P = pairs.shape[0]
    tc = np.zeros((P, 2))
    dtc = np.zeros((P, 2, 18))
    sg = np.zeros((P, 6), np.int8)
    fl = np.zeros(P, np.uint8)
    lib.ttie_oracle_eval(_ptr(x), _ptr(tri), _ptr(pairs), P, float(tc_scale),
                         _ptr(tc), _ptr(dtc), _ptr(sg), _ptr(fl))
    return tc, dtc, sg, fl


def filtered_sides(x, tri, pairs) -> np.ndarray:
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    pairs = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
    out = np.zeros((pairs.shape[0], 6), np.int8)
    lib.ttie_oracle_sides(_ptr(x), _ptr(tri), _ptr(pairs), pairs.shape[0], _ptr(out))
    return out


def evaluate(x, tri, pairs, tc_scale: float = 1.0, exact_active: bool = True) -> PairEval:
    tc, dtc, sg, fl = eval_pairs_f64(x, tri, pairs, tc_scale)
    if exact_active:
        act = exact.active_exact(x, tri, pairs, prefilter=filtered_sides(x, tri, pairs))
    else:
        act = (fl & 4) != 0
    return PairEval(np.asarray(pairs, np.int64).reshape(-1, 2), tc, dtc, sg, fl, act)


def gradient(ev: PairEval) -> np.ndarray:
    """Eq. 3: dT = 2 t0 t1^2 d t0 + 2 t1 t0^2 d t1 per pair ([P,18]; zero on inactive pairs)."""
    a, b = ev.tc[:, 0], ev.tc[:, 1]
    g = (2 * a * b * b)[:, None] * ev.dtc[:, 0] + (2 * b * a * a)[:, None] * ev.dtc[:, 1]
    return np.where(ev.active[:, None], g, 0.0)


def hessian_parts(ev: PairEval):
    """The three parts of Eq. 4 per pair ([P,18,18] each)."""
    a, b = ev.tc[:, 0], ev.tc[:, 1]
    u, v = ev.dtc[:, 0], ev.dtc[:, 1]
    uu = np.einsum("pi,pj->pij", u, u)
    vv = np.einsum("pi,pj->pij", v, v)
    vu = np.einsum("pi,pj->pij", v, u)
    uv = np.einsum("pi,pj->pij", u, v)
    p1 = (2 * b * b)[:, None, None] * uu
    p2 = (2 * a * a)[:, None, None] * vv
    p3 = (4 * a * b)[:, None, None] * (vu + uv)
    return p1, p2, p3


def hessian_inexact(ev: PairEval) -> np.ndarray:
    p1, p2, p3 = hessian_parts(ev)
    return np.where(ev.active[:, None, None], p1 + p2 + p3, 0.0)


def clamp_psd(M: np.ndarray) -> np.ndarray:
    """Symmetric eigen-decomposition with negative eigenvalues set to zero (batched)."""
    w, Q = np.linalg.eigh(M)
    w = np.maximum(w, 0.0)
    return np.einsum("pik,pk,pjk->pij", Q, w, Q)


def hessian_psd(ev: PairEval, mode: str = "per_part") -> np.ndarray:
    """Eigen-analysis of §1.1: parts 1 and 2 have one non-negative eigenvalue each; part 3 can
    have a negative one.  'per_part' keeps parts 1, 2 and the clamped part 3; 'drop_cross'
    keeps parts 1 and 2; 'whole' clamps the sum."""
    p1, p2, p3 = hessian_parts(ev)
    if mode == "per_part":
        H = p1 + p2 + clamp_psd(p3)
    elif mode == "drop_cross":
        H = p1 + p2
    elif mode == "whole":
        H = clamp_psd(p1 + p2 + p3)
    else:
        raise ValueError(mode)
    return np.where(ev.active[:, None, None], H, 0.0)


def pair_hessian_vector(x, tri, pairs, v, tc_scale: float = 1.0, h: float | None = None,
                        rtol: float = 1e-7, max_halvings: int = 24) -> np.ndarray:
    """Exact Hessian of T times v, per listed pair ([P,18]): the derivative of the Eq. 3 pair
    gradient 2ab(b da + a db) along v, taken at fixed pairs by the fourth-order central
    difference D(h) = (8(g(h) - g(-h)) - (g(2h) - g(-2h))) / 12h.  This includes the second
    derivatives of t_c that Eq. 4 drops.

    The pair gradient is smooth only piecewise: the min/max selections of the interval end
    points and the cut case switch where two values tie.  A step that straddles such a switch
    gives a meaningless quotient, so each pair's step is halved until D(h) and D(h/2) agree to
    rtol (relative to the pair's largest entry, floored at 1e-3 of the largest entry over all
    pairs) plus their rounding, 1e-13 |g| / h; D(h/2) is returned.  h starts at 1e-4 of the mean edge length over max |v|."""
    x = np.asarray(x, np.float64)
    v = np.asarray(v, np.float64).reshape(x.shape)
    pairs = np.asarray(pairs, np.int64).reshape(-1, 2)
    if h is None:
        e = x[tri[:, [1, 2, 0]]] - x[tri]
        vmax = np.abs(v).max()
        h = 1e-4 * float(np.linalg.norm(e, axis=-1).mean()) / (vmax if vmax > 0 else 1.0)

    def g(sub, t):
        tc, dtc, _, _ = eval_pairs_f64(x + t * v, tri, sub, tc_scale)
        a, b = tc[:, 0], tc[:, 1]
        return (2 * a * b)[:, None] * (b[:, None] * dtc[:, 0] + a[:, None] * dtc[:, 1])

    def D(sub, step):
        return (8 * (g(sub, step) - g(sub, -step)) - (g(sub, 2 * step) - g(sub, -2 * step))) / (12 * step)

    out = np.zeros((len(pairs), 18))
    if len(pairs) == 0:
        return out
    g0 = np.abs(g(pairs, 0.0)).max(1)       # rounding of D(h) is about eps * |g| / h
    todo = np.arange(len(pairs))
    prev = D(pairs, h)
    floor = None
    for _ in range(max_halvings):
        h *= 0.5
        cur = D(pairs[todo], h)
        if floor is None:
            floor = 1e-3 * np.abs(cur).max()
        scale = np.maximum(np.abs(cur).max(1), floor)
        ok = np.abs(cur - prev).max(1) <= rtol * scale + 1e-13 * g0[todo] / h
        out[todo[ok]] = cur[ok]
        todo, prev = todo[~ok], cur[~ok]
        if len(todo) == 0:
            return out
    raise ArithmeticError("pair_hessian_vector: no converged step for pairs %s" % pairs[todo[:8]].tolist())


def hessian_vector_product(x, tri, ev: PairEval, v, tc_scale: float = 1.0, h: float | None = None) -> np.ndarray:
    """[V,3]: sum over the intersecting pairs of ev of the exact pair Hessian times v."""
    act = np.nonzero(ev.active)[0]
    out = np.zeros((np.asarray(x).shape[0], 3))
    if len(act) == 0:
        return out
    hv = pair_hessian_vector(x, tri, ev.pairs[act], v, tc_scale, h)
    vid = pair_dofs(tri, ev.pairs[act])
    for r in range(6):
        np.add.at(out, vid[:, r], hv[:, 3 * r:3 * r + 3])
    return out


# ------------------------------------------------------------------ assembly
def pair_dofs(tri, pairs) -> np.ndarray:
    """[P,6] vertex ids of [A0 A1 A2 B0 B1 B2]."""
    return np.concatenate([tri[pairs[:, 0]], tri[pairs[:, 1]]], axis=1)


def assemble(tri, ev: PairEval, V: int, psd: str = "per_part"):
    """Sum per-pair gradients into a [V,3] array and per-pair Hessian 3x3 vertex blocks into a
    dict {(row_vertex, col_vertex): 3x3}.  Only active pairs contribute blocks; the block
    pattern is the union of the 6x6 vertex blocks of the active pairs."""
    act = np.nonzero(ev.active)[0]
    g = gradient(ev)
    grad = np.zeros((V, 3))
    blocks = {}
    if len(act) == 0:
        return grad, blocks
    H = hessian_psd(PairEval(ev.pairs[act], ev.tc[act], ev.dtc[act], ev.sides64[act],
                             ev.flags64[act], ev.active[act]), psd)
    vid = pair_dofs(tri, ev.pairs[act])
    for k, p in enumerate(act):
        for r in range(6):
            grad[vid[k, r]] += g[p, 3 * r:3 * r + 3]
            for c in range(6):
                key = (int(vid[k, r]), int(vid[k, c]))
                blk = H[k, 3 * r:3 * r + 3, 3 * c:3 * c + 3]
                if key in blocks:
                    blocks[key] = blocks[key] + blk
                else:
                    blocks[key] = blk.copy()
    return grad, blocks


def blocks_to_dense(blocks, verts):
    """Dense matrix over the listed vertices (3 DOFs each) from a block dict."""
    pos = {int(v): k for k, v in enumerate(verts)}
    n = len(verts)
    M = np.zeros((3 * n, 3 * n))
    for (r, c), b in blocks.items():
        M[3 * pos[r]:3 * pos[r] + 3, 3 * pos[c]:3 * pos[c] + 3] += b
    return M


# ------------------------------------------------------------------ solve
@dataclass
class NewtonParams:
    tc_scale: float = 1.0
    psd: str = "per_part"
    mu_rel: float = 1e-3          # mu = mu_rel * mean diagonal of H+ on active DOFs
    armijo_c: float = 1e-4
    ls_max_halvings: int = 20
    newton_max_it: int = 200
    push_eta: float = 0.5         # first trial step 1 + eta (overshoot past touching)
    max_step: float = 1.0         # largest vertex move per iteration, in mean edge lengths (0: none)
    mode: str = "self"
    ls_rule: str = "armijo"       # "armijo": Armijo or no pair; "fewer": also fewer pairs, E not above
    push_eta_max: float = 1.5     # "fewer": the overshoot doubles up to this while it leaves the count


def energy(x, tri, group, prm: NewtonParams):
    pairs = candidate_pairs(x, tri, group, prm.mode)
    ev = evaluate(x, tri, pairs, prm.tc_scale)
    return float(ev.T.sum()), int(ev.active.sum())


def newton_direction(x, tri, group, prm: NewtonParams):
    """One Newton system at x: returns (E, n_active, grad [V,3], d [V,3], active vertices)."""
    V = x.shape[0]
    pairs = candidate_pairs(x, tri, group, prm.mode)
    ev = evaluate(x, tri, pairs, prm.tc_scale)
    E, n_act = float(ev.T.sum()), int(ev.active.sum())
    grad, blocks = assemble(tri, ev, V, prm.psd)
    d = np.zeros((V, 3))
    if n_act == 0:
        return E, 0, grad, d, np.zeros(0, np.int64)
    verts = np.unique(pair_dofs(tri, ev.pairs[ev.active]))
    H = blocks_to_dense(blocks, verts)
    mu = prm.mu_rel * float(np.mean(np.diag(H)))
    rhs = -grad[verts].ravel()
    sol = np.linalg.solve(H + mu * np.eye(H.shape[0]), rhs)
    d[verts] = sol.reshape(-1, 3)
    return E, n_act, grad, d, verts


def line_search(x, d, E: float, slope: float, energy_at, prm: NewtonParams, n0: int | None = None,
                eta: float | None = None):
    """The backtracking line search of the Newton policy (reading of §1.2's unstated inexact
    Newton): trial steps 1 + eta (eta = push_eta unless given), then 1, 1/2, ...,
    2^-ls_max_halvings; the first trial with Armijo's condition E(x + a d) <= E + c a slope
    (slope = g.d < 0), or with no intersecting pair, or (rule "fewer", with n0 the pairs at x)
    with fewer intersecting pairs than n0 and E(x + a d) <= E, is taken, else the last.
    energy_at(xt) -> (E, intersecting pairs).  Returns (a, x + a d, E there, pairs there)."""
    eta = prm.push_eta if eta is None else eta
    for a in [1.0 + eta] + [0.5 ** k for k in range(prm.ls_max_halvings + 1)]:
        if a > 1.0 + eta:
            continue
        xt = x + a * d
        Et, nt = energy_at(xt)
        fewer = prm.ls_rule == "fewer" and n0 is not None and nt < n0 and Et <= E
        if nt == 0 or Et <= E + prm.armijo_c * a * slope or fewer:
            break
    return a, xt, Et, nt


def next_overshoot(eta: float, a: float, n0: int, n_new: int, prm: NewtonParams) -> float:
    """Rule "fewer": the overshoot of the next step.  A step that took the overshoot trial and
    left at least as many intersecting pairs doubles it (up to push_eta_max); a step that lowered
    the count returns it to push_eta."""
    if prm.ls_rule != "fewer":
        return prm.push_eta
    if n_new < n0:
        return prm.push_eta
    if a == 1.0 + eta and a > 1.0:
        return min(max(prm.push_eta_max, prm.push_eta), 2.0 * eta)
    return eta


def capped_direction(d, cap: float):
    """d scaled so that no vertex moves more than cap (0: no cap)."""
    dmax = float(np.linalg.norm(d, axis=1).max())
    return d * (cap / dmax) if cap > 0 and dmax > cap else d


def newton_solve(x0, tri, group=None, prm: NewtonParams | None = None, log=None):
    """Inexact Newton on E = sum T with a backtracking line search; stops when no pair
    intersects (decided exactly).  The direction is scaled so that no vertex moves more
    than max_step mean edge lengths (of the initial mesh) per iteration.

    The minimum T = 0 of a pair is reached at touching, which a Newton iteration on (ab)^2
    only approaches; so every iteration first tries the overshoot step 1 + eta, then
    1, 1/2, 1/4, ...  A trial is accepted when it satisfies Armijo's condition
    E(x + a d) <= E(x) + c a g.d or leaves no intersecting pair, or (rule "fewer") leaves
    fewer intersecting pairs without raising E; eta follows next_overshoot."""
    prm = prm or NewtonParams()
    x = np.array(x0, dtype=np.float64)
    edges = np.concatenate([x[tri[:, 1]] - x[tri[:, 0]], x[tri[:, 2]] - x[tri[:, 1]], x[tri[:, 0]] - x[tri[:, 2]]])
    cap = prm.max_step * float(np.linalg.norm(edges, axis=1).mean())
    eta = prm.push_eta
    for it in range(prm.newton_max_it):
        E, n_act, grad, d, verts = newton_direction(x, tri, group, prm)
        if log is not None:
            log.append((it, E, n_act))
        if n_act == 0:
            return x, it, True
        d = capped_direction(d, cap)
        a, x, _, nt = line_search(x, d, E, float(np.sum(grad * d)), lambda xt: energy(xt, tri, group, prm), prm,
                                  n0=n_act, eta=eta)
        eta = next_overshoot(eta, a, n_act, nt, prm)
    return x, prm.newton_max_it, False


def certify(x, tri, group=None, mode="self") -> int:
    """Number of intersecting pairs at x, decided exactly (0 = intersection-free in the
    paper's sense: coplanar overlaps and touching contacts do not count)."""
    pairs = candidate_pairs(x, tri, group, mode)
    act = exact.active_exact(x, tri, pairs, prefilter=filtered_sides(x, tri, pairs))
    return int(act.sum())
