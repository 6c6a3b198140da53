"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every check uses a closed form
(Eq. 1-4 on hand-built pairs, the eigenvalues stated in §1.1), an independent
exact predicate (separating axes), finite differences, invariances, or a
brute-force recomputation.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import ttie_inputs as ti

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- closed form (Eq. 1, 2)
def test_closed_form_pairs():
    spec = json.load(open(os.path.join(GOLDEN, "closed_form_pairs.json")))
    for c in spec["cases"]:
        m = ti.closed_form_pair(c["a0"], c["a1"], c["b0"], c["b1"], c["h"])
        ev = O.evaluate(m.x, m.tri, np.array([[0, 1]]))
        assert bool(ev.active[0]) == c["active"], c["name"]
        assert ev.T[0] == pytest.approx(c["T"], rel=1e-12, abs=1e-15), c["name"]
        # the FP64 open-interval test agrees (touching ends compare exactly equal: h = 0.5 keeps
        # every coordinate, crossing and t dyadic)
        assert bool(ev.flags64[0] & 4) == c["active"], c["name"]
        if c["active"]:
            lo_a, hi_a = sorted([c["a0"], c["a1"]])
            lo_b, hi_b = sorted([c["b0"], c["b1"]])
            # D points along -x here, so (t_c^0, t_c^1) = -(b, a) of the x-axis intervals
            assert ev.tc[0, 0] * ev.tc[0, 1] == pytest.approx((lo_a - hi_b) * (hi_a - lo_b), rel=1e-12)
            # Sum of the four t about their mean is zero (origin A cancels); |I_c| is the sum of lengths
            assert ev.tc[0, 1] - ev.tc[0, 0] == pytest.approx((hi_a - lo_a) + (hi_b - lo_b), rel=1e-12)
            # The listing's line direction D = n_B x n_A (its first normal belongs to the second
            # triangle), by hand for this geometry: n_A = (A1 - A0) x (A2 - A0) = (0, 0, 4h(a0 - a1)),
            # n_B = (B1 - B0) x (B2 - B0) = (0, 4h(b1 - b0), 0), so n_B x n_A = -16h^2 (b1 - b0)(a1 - a0) x^
            # and D = sx x^.  The end points of the segments sit at x = a0, a1 and b0, b1, so each
            # t_c is fixed, not only their product and difference (the opposite direction maps
            # (t_c^0, t_c^1) to (-t_c^1, -t_c^0)).
            sx = -np.sign(c["a1"] - c["a0"]) * np.sign(c["b1"] - c["b0"])
            tA, tB = sorted([sx * c["a0"], sx * c["a1"]]), sorted([sx * c["b0"], sx * c["b1"]])
            assert ev.tc[0, 0] == pytest.approx(tA[0] - tB[1], rel=1e-12), c["name"]
            assert ev.tc[0, 1] == pytest.approx(tA[1] - tB[0], rel=1e-12), c["name"]


def test_appendix_half_scale():
    """The appendix's listing returns (t_a^0 - t_b^1)/2; tc_scale=0.5 reproduces it, T/16."""
    m = ti.closed_form_pair(-0.2, 0.5, 0.1, 0.9)
    e1 = O.evaluate(m.x, m.tri, np.array([[0, 1]]), tc_scale=1.0)
    e2 = O.evaluate(m.x, m.tri, np.array([[0, 1]]), tc_scale=0.5)
    assert np.allclose(e2.tc, 0.5 * e1.tc)
    assert e2.T[0] == pytest.approx(e1.T[0] / 16)
    # the scale is a constant factor of t_c, so their gradients scale with it
    assert np.allclose(e2.dtc, 0.5 * e1.dtc) and np.abs(e1.dtc).max() > 0


def test_vertex_on_plane_case():
    """Signs (+,-,0): the cut segment runs from the on-plane vertex to the opposite edge."""
    h = 0.5
    # A in z=0, cut by y=0 in [-0.25, 0.5]
    A = [[0.0, -h, 0.0], [-0.5, h, 0.0], [1.0, h, 0.0]]
    # B in y=0 with one vertex on z=0 at x=0.75, others at z=+h (x=0) and z=-h (x=0.5):
    # its cut by z=0 is [0.25, 0.75]
    B = [[0.75, 0.0, 0.0], [0.0, 0.0, h], [0.5, 0.0, -h]]
    x = np.array(A + B)
    tri = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    ev = O.evaluate(x, tri, np.array([[0, 1]]))
    assert ev.active[0]
    assert ev.T[0] == pytest.approx(((-0.25 - 0.75) * (0.5 - 0.25)) ** 2, rel=1e-12)
    assert list(ev.sides64[0, :3]).count(0) == 1


# ----------------------------------------------------------------- exact predicate vs separating axes
def _sat_active(A, B):
    """Independent characterisation: the pair is intersecting iff no plane weakly separates the
    two triangles, i.e. their relative interiors meet and they are not coplanar.  The candidate
    axes (face normals, edge x edge) contain a facet normal of A (+) (-B), so checking them is
    complete.  Exact integer / rational arithmetic."""
    def sub(a, b):
        return [a[k] - b[k] for k in range(3)]

    def cross(a, b):
        return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]

    def dot(a, b):
        return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]
    ea = [sub(A[(k + 1) % 3], A[k]) for k in range(3)]
    eb = [sub(B[(k + 1) % 3], B[k]) for k in range(3)]
    axes = [cross(ea[0], ea[1]), cross(eb[0], eb[1])] + [cross(e, f) for e in ea for f in eb]
    for k in axes:
        if k == [0, 0, 0]:
            continue
        pa = [dot(k, p) for p in A]
        pb = [dot(k, p) for p in B]
        if max(pa) <= min(pb) or max(pb) <= min(pa):
            return False
    return True


@pytest.mark.parametrize("grid,seed", [(1, 0), (2, 1), (3, 2), (4, 3), (6, 4)])
def test_exact_matches_separating_axes_on_grid(grid, seed):
    m = ti.snapped_soup(90, seed, grid)
    pairs = np.array([(i, j) for i in range(m.F) for j in range(i + 1, m.F)], np.int64)
    act = O.exact.active_exact(m.x, m.tri, pairs)
    xi = m.x.astype(np.int64)
    ref = np.array([_sat_active([list(xi[v]) for v in m.tri[i]], [list(xi[v]) for v in m.tri[j]])
                    for i, j in pairs])
    assert np.array_equal(act, ref)
    # the grid makes every kind of case occur
    assert ref.sum() > 0 and (~ref).sum() > 0


def test_exact_matches_separating_axes_random():
    m = ti.triangle_soup(120, 11, size=0.5)
    pairs = np.array([(i, j) for i in range(m.F) for j in range(i + 1, m.F)], np.int64)
    act = O.exact.active_exact(m.x, m.tri, pairs, prefilter=O.filtered_sides(m.x, m.tri, pairs))
    xf = [[tuple(Fraction(float(c)) for c in v) for v in m.x[t]] for t in m.tri]
    ref = np.array([_sat_active([list(p) for p in xf[i]], [list(p) for p in xf[j]]) for i, j in pairs])
    assert np.array_equal(act, ref)
    assert ref.sum() > 50


def test_fp64_overlap_agrees_on_generic_pairs():
    """Away from degeneracies the listing's FP64 comparisons give the exact answer."""
    m = ti.triangle_soup(200, 5, size=0.5)
    pairs = np.array([(i, j) for i in range(m.F) for j in range(i + 1, m.F)], np.int64)
    ev = O.evaluate(m.x, m.tri, pairs)
    assert np.array_equal(ev.active, (ev.flags64 & 4) != 0)


# ----------------------------------------------------------------- certified side filter
def _exact_side(P, q):
    P = [[Fraction(float(c)) for c in p] for p in P]
    q = [Fraction(float(c)) for c in q]
    e1 = [P[1][k] - P[0][k] for k in range(3)]
    e2 = [P[2][k] - P[0][k] for k in range(3)]
    f = [q[k] - P[0][k] for k in range(3)]
    n = [e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]]
    d = n[0] * f[0] + n[1] * f[1] + n[2] * f[2]
    return (d > 0) - (d < 0)


def test_side_filter_never_wrong():
    rng = np.random.default_rng(7)
    base = ti.snapped_soup(150, 8, 3)
    # near-degenerate: integer grid plus perturbations of a few ulps
    x = base.x + rng.integers(-2, 3, base.x.shape) * np.ldexp(1.0, -50)
    x32 = (base.x + rng.normal(0, 1e-7, base.x.shape)).astype(np.float32).astype(np.float64)
    for xx in (base.x, x, x32):
        pairs = np.array([(i, j) for i in range(0, base.F, 3) for j in range(i + 1, base.F, 2)], np.int64)
        fs = O.filtered_sides(xx, base.tri, pairs)
        n_certain = 0
        for p, (i, j) in enumerate(pairs):
            A, B = xx[base.tri[i]], xx[base.tri[j]]
            ex = [_exact_side(A, b) for b in B] + [_exact_side(B, a) for a in A]
            for k in range(6):
                if fs[p, k] != 2:
                    n_certain += 1
                    assert fs[p, k] == ex[k]
        assert n_certain > 0


# ----------------------------------------------------------------- derivatives (Eq. 3, 4)
def _generic_active_pairs(seed=3, n=200, margin=0.05):
    m = ti.triangle_soup(n, seed, size=0.5)
    pairs = np.array([(i, j) for i in range(m.F) for j in range(i + 1, m.F)], np.int64)
    ev = O.evaluate(m.x, m.tri, pairs)
    keep = []
    for p in np.nonzero(ev.active)[0]:
        a, b = ev.tc[p]
        if min(abs(a), abs(b)) < margin:
            continue
        keep.append(p)
    return m, pairs[keep]


def _tc_at(m, pair, loc):
    x = m.x.copy()
    x[m.tri[pair[0]]] = loc[:9].reshape(3, 3)
    x[m.tri[pair[1]]] = loc[9:].reshape(3, 3)
    tc, dtc, _, fl = O.eval_pairs_f64(x, m.tri, pair[None, :])
    return tc[0], dtc[0], fl[0]


def _loc(m, pair):
    return np.concatenate([m.x[m.tri[pair[0]]].ravel(), m.x[m.tri[pair[1]]].ravel()])


def test_dual_gradient_matches_central_differences():
    m, pairs = _generic_active_pairs()
    assert len(pairs) >= 20
    h = 1e-6
    for pair in pairs[:40]:
        loc = _loc(m, pair)
        tc, dtc, fl = _tc_at(m, pair, loc)
        fd = np.zeros((2, 18))
        ok = True
        for k in range(18):
            e = np.zeros(18)
            e[k] = h
            tp, _, flp = _tc_at(m, pair, loc + e)
            tm, _, flm = _tc_at(m, pair, loc - e)
            ok &= (flp == fl) and (flm == fl)
            fd[:, k] = (tp - tm) / (2 * h)
        if not ok:
            continue
        assert np.allclose(dtc, fd, rtol=1e-5, atol=1e-7 * np.abs(dtc).max())


def _T_and_g(m, pair, loc):
    x = m.x.copy()
    x[m.tri[pair[0]]] = loc[:9].reshape(3, 3)
    x[m.tri[pair[1]]] = loc[9:].reshape(3, 3)
    ev = O.evaluate(x, m.tri, pair[None, :])
    return ev.T[0], O.gradient(ev)[0], ev


def test_eq3_gradient_is_gradient_of_T():
    m, pairs = _generic_active_pairs(seed=4)
    h = 1e-6
    for pair in pairs[:25]:
        loc = _loc(m, pair)
        T, g, _ = _T_and_g(m, pair, loc)
        fd = np.array([(_T_and_g(m, pair, loc + h * np.eye(18)[k])[0] -
                        _T_and_g(m, pair, loc - h * np.eye(18)[k])[0]) / (2 * h) for k in range(18)])
        assert np.allclose(g, fd, rtol=1e-5, atol=1e-8 * np.abs(g).max())


def test_eq4_is_exact_hessian_minus_dropped_terms():
    """Eq. 4 equals the exact Hessian of (ab)^2 minus 2ab(b d2a + a d2b) (§1.1, "ignoring the
    asymmetric part"); exact Hessian and d2a, d2b from central differences of the gradients."""
    m, pairs = _generic_active_pairs(seed=6)
    h = 1e-5
    for pair in pairs[:10]:
        loc = _loc(m, pair)
        T, g, ev = _T_and_g(m, pair, loc)
        a, b = ev.tc[0]
        Hfd = np.zeros((18, 18))
        d2a = np.zeros((18, 18))
        d2b = np.zeros((18, 18))
        for k in range(18):
            e = h * np.eye(18)[k]
            _, gp, evp = _T_and_g(m, pair, loc + e)
            _, gm, evm = _T_and_g(m, pair, loc - e)
            Hfd[:, k] = (gp - gm) / (2 * h)
            d2a[:, k] = (evp.dtc[0, 0] - evm.dtc[0, 0]) / (2 * h)
            d2b[:, k] = (evp.dtc[0, 1] - evm.dtc[0, 1]) / (2 * h)
        Hin = O.hessian_inexact(ev)[0]
        dropped = 2 * a * b * (b * d2a + a * d2b)
        scale = np.abs(Hfd).max()
        assert np.allclose(Hin, Hfd - dropped, atol=2e-5 * scale)


def test_eq4_symbolic_expansion():
    """sympy: Hessian of (a b)^2 = Eq. 4 + 2ab(b Hess a + a Hess b) for generic a(x), b(x)."""
    sp = pytest.importorskip("sympy")
    xs = sp.symbols("x0:3")
    a = sp.Function("a")(*xs)
    b = sp.Function("b")(*xs)
    T = (a * b) ** 2
    u = sp.Matrix([sp.diff(a, v) for v in xs])
    w = sp.Matrix([sp.diff(b, v) for v in xs])
    H = sp.hessian(T, xs)
    eq4 = 2 * b ** 2 * u * u.T + 2 * a ** 2 * w * w.T + 4 * a * b * (w * u.T + u * w.T)
    dropped = 2 * a * b * (b * sp.hessian(a, xs) + a * sp.hessian(b, xs))
    assert sp.simplify(H - eq4 - dropped) == sp.zeros(3, 3)


# ----------------------------------------------------------------- eigen-analysis (§1.1)
def test_eigenanalysis_closed_forms():
    m, pairs = _generic_active_pairs(seed=8)
    ev = O.evaluate(m.x, m.tri, pairs)
    p1, p2, p3 = O.hessian_parts(ev)
    a, b = ev.tc[:, 0], ev.tc[:, 1]
    u, v = ev.dtc[:, 0], ev.dtc[:, 1]
    for k in range(len(pairs)):
        w1 = np.linalg.eigvalsh(p1[k])
        w2 = np.linalg.eigvalsh(p2[k])
        # part 1 and part 2: a single non-zero eigenvalue 2 b^2 |du|^2, 2 a^2 |dv|^2
        assert w1[-1] == pytest.approx(2 * b[k] ** 2 * u[k] @ u[k], rel=1e-10)
        assert w2[-1] == pytest.approx(2 * a[k] ** 2 * v[k] @ v[k], rel=1e-10)
        assert np.abs(w1[:-1]).max() < 1e-10 * w1[-1]
        # part 3: trace is the paper's 8ab du.dv; its two eigenvalues 4ab(u.v +- |u||v|)
        assert np.trace(p3[k]) == pytest.approx(8 * a[k] * b[k] * u[k] @ v[k], rel=1e-10)
        w3 = np.linalg.eigvalsh(p3[k])
        nu, nv = np.linalg.norm(u[k]), np.linalg.norm(v[k])
        lo, hi = sorted([4 * a[k] * b[k] * (u[k] @ v[k] + nu * nv), 4 * a[k] * b[k] * (u[k] @ v[k] - nu * nv)])
        assert w3[0] == pytest.approx(lo, rel=1e-9) and w3[-1] == pytest.approx(hi, rel=1e-9)


def test_psd_projection_properties():
    m, pairs = _generic_active_pairs(seed=9)
    ev = O.evaluate(m.x, m.tri, pairs)
    Hp = O.hessian_psd(ev, "per_part")
    p3 = O.hessian_parts(ev)[2]
    a, b = ev.tc[:, 0], ev.tc[:, 1]
    u, v = ev.dtc[:, 0], ev.dtc[:, 1]
    for k in range(len(pairs)):
        H = Hp[k]
        assert np.allclose(H, H.T, atol=1e-14 * np.abs(H).max())
        w = np.linalg.eigvalsh(H)
        assert w[0] >= -1e-12 * w[-1]
        assert np.sum(w > 1e-10 * w[-1]) <= 2                       # rank <= 2
        for ax in range(3):                                           # translations are null
            t = np.zeros(18)
            t[ax::3] = 1.0
            assert np.abs(H @ t).max() <= 1e-9 * np.abs(H).max()
        # clamped part 3 = 2|ab||u||v| (u^ - v^)(u^ - v^)^T (its non-negative eigenpair)
        nu, nv = np.linalg.norm(u[k]), np.linalg.norm(v[k])
        wv = u[k] / nu - v[k] / nv
        closed = 2 * abs(a[k] * b[k]) * nu * nv * np.outer(wv, wv)
        assert np.allclose(O.clamp_psd(p3[k:k + 1])[0], closed, atol=1e-10 * np.abs(closed).max())
        # the default projection keeps parts 1 and 2 and that eigenpair of part 3 (per part, §1.1),
        # not the clamp of the sum, which has rank one: H+ = 2b^2 uu' + 2a^2 vv' + closed, rank 2
        per_part = 2 * b[k] ** 2 * np.outer(u[k], u[k]) + 2 * a[k] ** 2 * np.outer(v[k], v[k]) + closed
        assert np.allclose(H, per_part, atol=1e-10 * np.abs(per_part).max())
        assert np.sum(w > 1e-10 * w[-1]) == 2


# ----------------------------------------------------------------- invariances
def test_invariances():
    m, pairs = _generic_active_pairs(seed=10)
    rng = np.random.default_rng(0)
    R = ti.random_rotation(rng)
    t = rng.normal(size=3)
    for pair in pairs[:30]:
        x = m.x
        ev = O.evaluate(x, m.tri, pair[None, :])
        T0 = ev.T[0]
        # swap the triangles
        assert O.evaluate(x, m.tri, pair[::-1][None, :]).T[0] == pytest.approx(T0, rel=1e-9)
        # cyclic and odd permutations of a triangle's vertices
        for perm in ([1, 2, 0], [2, 0, 1], [0, 2, 1], [1, 0, 2]):
            tri2 = m.tri.copy()
            tri2[pair[0]] = m.tri[pair[0]][perm]
            assert O.evaluate(x, tri2, pair[None, :]).T[0] == pytest.approx(T0, rel=1e-9)
        # rigid motion and reflection
        assert O.evaluate(x @ R.T + t, m.tri, pair[None, :]).T[0] == pytest.approx(T0, rel=1e-8)
        assert O.evaluate(x * np.array([-1, 1, 1]), m.tri, pair[None, :]).T[0] == pytest.approx(T0, rel=1e-9)
        # scaling: T is homogeneous of degree 4
        assert O.evaluate(2.5 * x, m.tri, pair[None, :]).T[0] == pytest.approx(2.5 ** 4 * T0, rel=1e-9)
        # per-pair gradient: zero net force and zero net torque
        g = O.gradient(ev)[0].reshape(6, 3)
        X = np.concatenate([x[m.tri[pair[0]]], x[m.tri[pair[1]]]])
        sc = np.abs(g).max() * (1 + np.abs(X).max())
        assert np.abs(g.sum(0)).max() < 1e-10 * sc
        assert np.abs(np.cross(X, g).sum(0)).max() < 1e-10 * sc


# ----------------------------------------------------------------- pairs, assembly, solve
def test_candidate_pairs_brute_force_loops():
    m = ti.cloth(9, seed=2)
    lo, hi = m.x[m.tri].min(1), m.x[m.tri].max(1)
    ref = []
    for i in range(m.F):
        for j in range(i + 1, m.F):
            if set(m.tri[i]) & set(m.tri[j]):
                continue
            if all(lo[i][k] <= hi[j][k] and lo[j][k] <= hi[i][k] for k in range(3)):
                ref.append((i, j))
    got = O.candidate_pairs(m.x, m.tri)
    assert [tuple(p) for p in got] == ref
    for i in (0, 7, 50):
        row = sorted([j for (a, j) in ref if a == i] + [a for (a, j) in ref if j == i])
        assert list(O.partners_of(m.x, m.tri, i)) == row


def test_partners_of_rows_in_every_mode():
    """Brute-force rows (closed boxes, no shared vertex, the mode's group rule) against
    partners_of in the three pair modes."""
    m = ti.two_icospheres(offset=(1.6, 0.0, 0.0))
    lo, hi = m.x[m.tri].min(1), m.x[m.tri].max(1)
    for mode in ("self", "inter", "instance"):
        for i in (0, 17, 200, 333, 639):
            row = []
            for j in range(m.F):
                if j == i or set(m.tri[i]) & set(m.tri[j]):
                    continue
                if mode == "inter" and m.group[i] == m.group[j]:
                    continue
                if mode == "instance" and m.group[i] != m.group[j]:
                    continue
                if all(lo[i][k] <= hi[j][k] and lo[j][k] <= hi[i][k] for k in range(3)):
                    row.append(j)
            assert list(O.partners_of(m.x, m.tri, i, m.group, mode)) == row, (mode, i)


def test_certify_respects_pair_mode():
    """Two intersecting closed-form pairs, each inside one group, and one pair across groups:
    the count in each mode is the hand count."""
    a = ti.closed_form_pair(-0.2, 0.5, 0.1, 0.9)               # intersects (Eq. 1 closed form)
    x = np.concatenate([a.x, a.x + [10.0, 0.0, 0.0], a.x + [20.0, 0.0, 0.0]])
    tri = np.concatenate([a.tri, a.tri + 6, a.tri + 12]).astype(np.int32)
    group = np.array([0, 0, 1, 1, 2, 3], np.int32)
    assert O.certify(x, tri, group, "self") == 3
    assert O.certify(x, tri, group, "instance") == 2
    assert O.certify(x, tri, group, "inter") == 1
    # the energy of the line search counts the same pairs (three copies of one pair: T each)
    T1 = O.energy(a.x, a.tri, None, O.NewtonParams())[0]
    for mode, k in (("self", 3), ("instance", 2), ("inter", 1)):
        E, n = O.energy(x, tri, group, O.NewtonParams(mode=mode))
        assert n == k and E == pytest.approx(k * T1, rel=1e-12), mode


def test_pair_modes():
    m = ti.two_icospheres()
    inter = O.candidate_pairs(m.x, m.tri, m.group, "inter", aabb=False)
    assert len(inter) == 320 * 320
    assert np.all(m.group[inter[:, 0]] != m.group[inter[:, 1]])
    inst = O.candidate_pairs(m.x, m.tri, m.group, "instance")
    assert np.all(m.group[inst[:, 0]] == m.group[inst[:, 1]])


def test_assembly_matches_dense_scatter():
    m = ti.cloth(12, seed=21)
    pairs = O.candidate_pairs(m.x, m.tri)
    ev = O.evaluate(m.x, m.tri, pairs)
    assert ev.active.sum() > 3
    grad, blocks = O.assemble(m.tri, ev, m.V)
    g = O.gradient(ev)
    H = O.hessian_psd(ev)
    Gd = np.zeros(3 * m.V)
    Hd = np.zeros((3 * m.V, 3 * m.V))
    dof = O.pair_dofs(m.tri, ev.pairs)
    for p in range(len(pairs)):
        idx = (3 * dof[p][:, None] + np.arange(3)[None, :]).ravel()
        Gd[idx] += g[p]
        Hd[np.ix_(idx, idx)] += H[p]
    assert np.allclose(grad.ravel(), Gd)
    M = O.blocks_to_dense(blocks, np.arange(m.V))
    assert np.allclose(M, Hd)
    pattern = {(int(r), int(c)) for p in np.nonzero(ev.active)[0] for r in dof[p] for c in dof[p]}
    assert set(blocks) == pattern


def test_newton_direction_solves_system():
    m = ti.cloth(12, seed=21)
    prm = O.NewtonParams()
    E, n, grad, d, verts = O.newton_direction(m.x, m.tri, None, prm)
    assert n > 0 and E > 0
    pairs = O.candidate_pairs(m.x, m.tri)
    ev = O.evaluate(m.x, m.tri, pairs)
    _, blocks = O.assemble(m.tri, ev, m.V)
    H = O.blocks_to_dense(blocks, verts)
    mu = prm.mu_rel * np.mean(np.diag(H))
    r = (H + mu * np.eye(len(H))) @ d[verts].ravel() + grad[verts].ravel()
    assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(grad)
    assert np.sum(grad * d) < 0   # descent direction


def test_newton_rows_are_vertices_of_intersecting_pairs():
    """The policy's system (H+ + mu I) d = -g lives on the vertices of intersecting pairs, and
    mu is mu_rel times the mean diagonal there (reading 10): no vertex of a candidate that
    does not intersect is a row."""
    m = ti.triangle_soup(120, seed=5, size=0.45)
    prm = O.NewtonParams()
    pairs = O.candidate_pairs(m.x, m.tri)
    act = O.exact.active_exact(m.x, m.tri, pairs)
    assert 0 < act.sum() < len(pairs)
    rows = sorted({int(v) for p in pairs[act] for t in p for v in m.tri[t]})
    _, n, _, d, verts = O.newton_direction(m.x, m.tri, None, prm)
    assert n == act.sum() and list(verts) == rows
    others = np.setdiff1d(np.arange(m.V), rows)
    assert np.all(d[others] == 0.0)


def test_mesh_edges_counts():
    """Unique undirected edges: 3F/2 on a closed mesh (every edge shared by two triangles),
    V + F - 1 on a triangulated disk (Euler: V - E + F = 1)."""
    s = ti.icosphere(2)
    e = O.mesh_edges(s.tri)
    assert len(e) == 3 * s.F // 2 and np.all(e[:, 0] < e[:, 1])
    c = ti.cloth(9, seed=2, crossing=False)
    assert len(O.mesh_edges(c.tri)) == c.V + c.F - 1
    assert len({tuple(r) for r in O.mesh_edges(c.tri)}) == c.V + c.F - 1


def test_side_filter_certifies_generic_signs():
    """The FP64 side filter leaves a sign undecided only near a tie: on random triangles every
    one of the six signs of almost every pair is certified."""
    m = ti.triangle_soup(150, seed=11, size=0.5)
    pairs = np.array([(i, j) for i in range(m.F) for j in range(i + 1, m.F)], np.int64)
    f = O.filtered_sides(m.x, m.tri, pairs)
    assert np.mean(f == 2) < 1e-3
    for k in range(6):
        assert np.mean(f[:, k] == 2) < 1e-3, k


def test_line_search_rule():
    """The policy's line search on E(x) = |x|^2 (one intersecting pair throughout unless stated),
    decided by hand: trials 1.5, 1, 1/2, ...; Armijo E(x + a d) <= E + c a g.d, or no pair."""
    prm = O.NewtonParams(armijo_c=1e-4, push_eta=0.5, ls_max_halvings=4)
    x = np.array([[1.0, 0.0, 0.0]])
    E, g = 1.0, 2 * x
    quad = lambda xt: (float(np.sum(xt * xt)), 1)
    # d = -x: 1.5 lands at -0.5 x, E = 0.25 <= 1 - 1.5e-4 * 2: the overshoot is taken
    d = -x
    a, xt, Et, _ = O.line_search(x, d, E, float(np.sum(g * d)), quad, prm)
    assert a == 1.5 and Et == pytest.approx(0.25)
    # d = -2x: 1.5 gives E = 4, 1 gives E = 1 (no decrease, rejected), 1/2 gives 0
    d = -2 * x
    a, xt, Et, _ = O.line_search(x, d, E, float(np.sum(g * d)), quad, prm)
    assert a == 0.5 and Et == 0.0
    # no intersecting pair accepts the first trial whatever its energy
    a, _, _, nt = O.line_search(x, d, E, float(np.sum(g * d)), lambda xt: (100.0, 0), prm)
    assert a == 1.5 and nt == 0
    # nothing acceptable: the last trial, 2^-4, is taken
    a, _, _, _ = O.line_search(x, x, E, float(np.sum(g * x)), quad, prm)
    assert a == 0.5 ** 4
    # rule "fewer": a trial with fewer intersecting pairs and no higher energy is accepted even
    # without Armijo's decrease (E(x + a d) = E at every trial here); with as many pairs it is not
    flat = lambda cnt: (lambda xt: (E, cnt))
    prm_f = O.NewtonParams(armijo_c=1e-4, push_eta=0.5, ls_max_halvings=4, ls_rule="fewer")
    a, _, _, nt = O.line_search(x, -x, E, -2.0, flat(1), prm_f, n0=2)
    assert a == 1.5 and nt == 1
    a, _, _, _ = O.line_search(x, -x, E, -2.0, flat(2), prm_f, n0=2)
    assert a == 0.5 ** 4
    # ... and not under the Armijo-only rule
    prm_a = O.NewtonParams(armijo_c=1e-4, push_eta=0.5, ls_max_halvings=4, ls_rule="armijo")
    a, _, _, _ = O.line_search(x, -x, E, -2.0, flat(1), prm_a, n0=2)
    assert a == 0.5 ** 4
    # a larger overshoot is the first trial
    a, _, _, _ = O.line_search(x, -x, E, -2.0, flat(1), prm_f, n0=2, eta=3.0)
    assert a == 4.0


def test_adaptive_overshoot():
    """Rule "fewer": the overshoot doubles after a step that took it and left as many pairs, up
    to push_eta_max, and returns to push_eta when the count falls; other steps keep it."""
    prm = O.NewtonParams(push_eta=0.5, push_eta_max=7.0, ls_rule="fewer")
    assert O.next_overshoot(0.5, 1.5, 12, 12, prm) == 1.0
    assert O.next_overshoot(4.0, 5.0, 12, 13, prm) == 7.0
    assert O.next_overshoot(7.0, 8.0, 12, 12, prm) == 7.0
    assert O.next_overshoot(4.0, 5.0, 12, 11, prm) == 0.5
    assert O.next_overshoot(4.0, 1.0, 12, 12, prm) == 4.0
    assert O.next_overshoot(4.0, 5.0, 12, 12, O.NewtonParams(push_eta=0.5, ls_rule="armijo")) == 0.5


def test_step_cap_bounds_each_iteration():
    """No vertex moves more than (1 + push_eta) max_step mean edge lengths in one iteration
    (the largest trial of the capped direction)."""
    m = ti.two_icospheres(offset=(1.95, 0.0, 0.0))
    prm = O.NewtonParams(newton_max_it=1, mode="inter", max_step=0.05)
    e = np.concatenate([m.x[m.tri[:, 1]] - m.x[m.tri[:, 0]], m.x[m.tri[:, 2]] - m.x[m.tri[:, 1]],
                        m.x[m.tri[:, 0]] - m.x[m.tri[:, 2]]])
    cap = prm.max_step * float(np.linalg.norm(e, axis=1).mean())
    _, _, _, d, _ = O.newton_direction(m.x, m.tri, m.group, prm)
    assert np.linalg.norm(d, axis=1).max() > cap          # the cap is active here
    x1, _, _ = O.newton_solve(m.x, m.tri, m.group, prm)
    moved = np.linalg.norm(x1 - m.x, axis=1).max()
    assert 0 < moved <= (1 + prm.push_eta) * cap * (1 + 1e-12)
    dc = O.capped_direction(d, cap)
    assert np.linalg.norm(dc, axis=1).max() == pytest.approx(cap)
    assert np.allclose(dc / np.linalg.norm(dc), d / np.linalg.norm(d))


@pytest.mark.slow
@pytest.mark.parametrize("case", ["spheres_shallow", "cloth_mild"])
def test_newton_solve_reaches_intersection_free(case):
    if case == "spheres_shallow":
        m, mode = ti.two_icospheres(offset=(1.95, 0.0, 0.0)), "inter"
    else:
        m, mode = ti.cloth(16, seed=2, shear=0.05), "self"
    assert O.certify(m.x, m.tri, m.group, mode) > 0
    x, it, ok = O.newton_solve(m.x, m.tri, m.group, O.NewtonParams(newton_max_it=30, mode=mode))
    assert ok
    assert O.certify(x, m.tri, m.group, mode) == 0


# ----------------------------------------------------------------- exact Hessian-vector product
def _hvp_case(seed=3):
    m = ti.triangle_soup(200, seed, size=0.5)
    pairs = O.candidate_pairs(m.x, m.tri)
    ev = O.evaluate(m.x, m.tri, pairs)
    g, _ = O.assemble(m.tri, ev, m.V)
    return m, ev, g


def test_hvp_euler_identity():
    """T is homogeneous of degree 4 in the positions (t_c are lengths, Eq. 1), so H x = 3 g."""
    m, ev, g = _hvp_case()
    assert ev.active.sum() > 20
    v = m.x - m.x.mean(0)
    hv = O.hessian_vector_product(m.x, m.tri, ev, v)
    assert np.allclose(hv, 3 * g, rtol=0, atol=1e-7 * np.abs(g).max())


def test_hvp_rotation_and_translation():
    """T is invariant under rigid motions: H (w x x) = w x g per vertex and H c = 0."""
    m, ev, g = _hvp_case(seed=5)
    rng = np.random.default_rng(0)
    w = rng.normal(size=3)
    hv = O.hessian_vector_product(m.x, m.tri, ev, np.cross(w, m.x))
    assert np.allclose(hv, np.cross(w, g), rtol=0, atol=1e-7 * np.abs(g).max() * np.abs(w).max())
    c = rng.normal(size=3)
    ht = O.hessian_vector_product(m.x, m.tri, ev, np.tile(c, (m.V, 1)))
    r = m.x - m.x.mean(0)
    h_unit = 3 * np.abs(g).max() / np.abs(r).max()      # |H| from Euler's identity, H r = 3 g
    assert np.abs(ht).max() < 1e-6 * h_unit * np.abs(c).max()
    # the inexact Hessian of Eq. 4 is not rotation-consistent: the pin tells them apart
    act = np.nonzero(ev.active)[0]
    H = O.hessian_inexact(ev)[act]
    vid = O.pair_dofs(m.tri, ev.pairs[act])
    u = np.cross(w, m.x)[vid].reshape(len(act), 18)
    hin = np.zeros_like(m.x)
    for r in range(6):
        np.add.at(hin, vid[:, r], np.einsum("pij,pj->pi", H, u)[:, 3 * r:3 * r + 3])
    assert np.abs(hin - np.cross(w, g)).max() > 1e-3 * np.abs(g).max()


def test_hvp_quadratic_form_and_symmetry():
    """v.Hv is the second difference of E along v (T values only); u.Hv = v.Hu."""
    m, ev, g = _hvp_case(seed=7)
    rng = np.random.default_rng(1)
    v = rng.normal(size=m.x.shape)
    u = rng.normal(size=m.x.shape)
    act = ev.pairs[ev.active]

    def E(xx):
        tc, _, _, _ = O.eval_pairs_f64(xx, m.tri, act)
        return float(((tc[:, 0] * tc[:, 1]) ** 2).sum())

    eps = 1e-6   # well inside the smooth piece of every pair (the interval end points have kinks)
    d2 = (E(m.x + eps * v) - 2 * E(m.x) + E(m.x - eps * v)) / eps ** 2
    hv = O.hessian_vector_product(m.x, m.tri, ev, v)
    hu = O.hessian_vector_product(m.x, m.tri, ev, u)
    assert float((v * hv).sum()) == pytest.approx(d2, rel=1e-5)
    assert float((u * hv).sum()) == pytest.approx(float((v * hu).sum()), rel=1e-5)


def test_psd_whole_and_drop_cross_projections():
    """'whole' is the projection of Eq. 4 onto the PSD cone: H+ is PSD, H+ - H is PSD and
    H+ (H+ - H) = 0 (complementarity); Eq. 4 has inertia (1, 1, 16), so H+ has rank one.
    'drop_cross' is parts 1 + 2 exactly."""
    m, pairs = _generic_active_pairs(seed=9)
    ev = O.evaluate(m.x, m.tri, pairs)
    H = O.hessian_inexact(ev)
    Hw = O.hessian_psd(ev, "whole")
    p1, p2, _ = O.hessian_parts(ev)
    assert np.array_equal(O.hessian_psd(ev, "drop_cross"), p1 + p2)
    for k in range(len(pairs)):
        s = np.abs(H[k]).max()
        w = np.linalg.eigvalsh(H[k])
        assert (w > 1e-9 * s).sum() == 1 and (w < -1e-9 * s).sum() == 1
        assert np.linalg.eigvalsh(Hw[k]).min() >= -1e-12 * s
        D = Hw[k] - H[k]
        assert np.linalg.eigvalsh(D).min() >= -1e-12 * s
        assert np.abs(Hw[k] @ D).max() <= 1e-10 * s * s
        assert np.linalg.matrix_rank(Hw[k], tol=1e-9 * s) == 1


def test_energy_jumps_at_vertex_face_contact():
    """Eq. 1-2 measure the overlap of the two intervals on the planes' common line, not a depth:
    when a vertex of A passes through the interior of B, A's interval is born as a point inside
    B's interval, so T jumps from 0 to about (half the chord of B)^4 instead of growing from 0.
    T is smooth inside the intersecting set but not continuous across this part of its border
    (it is continuous where the intervals separate: t_c^0 or t_c^1 -> 0)."""
    B = np.array([[-1.0, -1.0, 0.0], [1.5, -1.0, 0.0], [-1.0, 1.5, 0.0]])
    tri = np.array([[0, 1, 2], [3, 4, 5]])
    T = {}
    for eps in [1e-9, 0.0, -1e-9, -1e-6]:
        A = np.array([[0.0, 0.0, eps], [0.3, 0.1, 1.0], [-0.1, 0.3, 1.0]])
        ev = O.evaluate(np.concatenate([A, B]), tri, np.array([[0, 1]]))
        T[eps] = float(ev.T[0])
    assert T[1e-9] == 0.0 and T[0.0] == 0.0
    assert T[-1e-9] > 1.0 and T[-1e-6] == pytest.approx(T[-1e-9], rel=1e-5)


# ----------------------------------------------------------------- elastic term (quasi-static simulation)
def _spring_case(seed=8, anchors=True):
    m = ti.cloth(6, seed=seed, shear=0.0)
    rng = np.random.default_rng(seed)
    el = O.springs_at_rest(m.x, m.tri, k_edge=2.5)
    x = m.x + 0.05 * rng.standard_normal(m.x.shape)
    if anchors:
        el.anchors = np.array([0, 5, 17])
        el.targets = m.x[el.anchors] + 0.1 * rng.standard_normal((3, 3))
        el.k_anchor = 0.7
    return m, el, x


def test_spring_closed_form():
    k, L, dl = 3.0, 0.4, 0.05
    x = np.array([[0.0, 0.0, 0.0], [L + dl, 0.0, 0.0]])
    el = O.Elastic(np.array([[0, 1]]), np.array([L]), k)
    assert O.elastic_energy(x, el) == pytest.approx(0.5 * k * dl * dl, rel=1e-13)
    g = O.elastic_gradient(x, el)
    assert np.allclose(g, [[-k * dl, 0, 0], [k * dl, 0, 0]], rtol=1e-13, atol=1e-15)
    x[1, 0] = L
    assert O.elastic_energy(x, el) == 0.0 and not O.elastic_gradient(x, el).any()
    # an anchor: k_a/2 |x - t|^2
    el = O.Elastic(np.zeros((0, 2), np.int64), np.zeros(0), 0.0, np.array([1]), np.array([[0.0, 0.3, 0.4]]), 2.0)
    assert O.elastic_energy(x, el) == pytest.approx(0.5 * 2.0 * (L * L + 0.25), rel=1e-13)
    assert np.allclose(O.elastic_gradient(x, el)[1], 2.0 * (x[1] - [0.0, 0.3, 0.4]))


def test_elastic_gradient_central_differences():
    m, el, x = _spring_case()
    g = O.elastic_gradient(x, el)
    h = 1e-6
    rng = np.random.default_rng(1)
    for v in rng.choice(m.V, 12, replace=False):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, a] += h
            xm[v, a] -= h
            fd = (O.elastic_energy(xp, el) - O.elastic_energy(xm, el)) / (2 * h)
            assert fd == pytest.approx(g[v, a], rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("stretch", [1.3, 0.6])
def test_spring_hessian_central_differences(stretch):
    rng = np.random.default_rng(2)
    xi, n = rng.standard_normal(3), rng.standard_normal(3)
    L, k = 0.8, 1.7
    xj = xi + stretch * L * n / np.linalg.norm(n)
    el = O.Elastic(np.array([[0, 1]]), np.array([L]), k)
    x = np.stack([xi, xj])
    H = O.spring_hessian(xi, xj, L, k)
    h = 1e-6
    fd = np.zeros((6, 6))
    for c in range(6):
        xp, xm = x.copy(), x.copy()
        xp.ravel()[c] += h
        xm.ravel()[c] -= h
        fd[:, c] = (O.elastic_gradient(xp, el) - O.elastic_gradient(xm, el)).ravel() / (2 * h)
    assert np.allclose(H, fd, rtol=1e-6, atol=1e-7 * k)


@pytest.mark.parametrize("stretch", [1.3, 0.6])
def test_projected_spring_spectrum(stretch):
    """[[K,-K],[-K,K]] has twice K's eigenvalues and three zeros; K has k along the spring and
    k (1 - L/l) twice across it, so the projection keeps 2k and 2k max(0, 1 - L/l) (twice)."""
    rng = np.random.default_rng(3)
    xi, n = rng.standard_normal(3), rng.standard_normal(3)
    L, k = 0.8, 1.7
    xj = xi + stretch * L * n / np.linalg.norm(n)
    w = np.sort(np.linalg.eigvalsh(O.clamp_psd(O.spring_hessian(xi, xj, L, k)[None])[0]))
    t = 2 * k * max(0.0, 1 - 1 / stretch)
    assert np.allclose(w, np.sort([2 * k, t, t, 0, 0, 0]), atol=1e-12 * k)


def test_elastic_invariances():
    m, el, x = _spring_case(anchors=False)
    E = O.elastic_energy(x, el)
    assert O.elastic_energy(x + np.array([0.3, -1.0, 2.0]), el) == pytest.approx(E, rel=1e-12)
    R = ti.random_rotation(np.random.default_rng(4))
    assert O.elastic_energy(x @ R.T, el) == pytest.approx(E, rel=1e-12)
    assert np.abs(O.elastic_gradient(x, el).sum(axis=0)).max() <= 1e-12 * np.abs(O.elastic_gradient(x, el)).max()


def test_elastic_blocks_quadratic_form():
    """With every spring stretched the projection changes nothing, so v.Hv is the second central
    difference of E_el along v; the scatter into vertex blocks is checked by that alone."""
    m, el, x = _spring_case()
    x = m.x * 1.2   # every spring stretched by 20 %
    M = O.blocks_to_dense(O.elastic_blocks(x, el), np.arange(m.V))
    v = np.random.default_rng(5).standard_normal(x.shape)
    h = 1e-4
    d2 = (O.elastic_energy(x + h * v, el) - 2 * O.elastic_energy(x, el) + O.elastic_energy(x - h * v, el)) / (h * h)
    # E_el is a polynomial of degree 2 in l: fourth-order terms of the difference stay below 1e-6
    assert v.ravel() @ M @ v.ravel() == pytest.approx(d2, rel=1e-6)
    assert np.linalg.eigvalsh(O.blocks_to_dense(O.elastic_blocks(_spring_case()[2], el), np.arange(m.V))).min() >= -1e-10


def test_newton_direction_elastic_solves_system():
    m = ti.cloth(12, seed=21)
    prm = O.NewtonParams()
    el = O.springs_at_rest(m.x, m.tri, k_edge=1e-3)
    E, n, grad, d, rows = O.newton_direction_elastic(m.x, m.tri, None, prm, el)
    assert n > 0
    pairs = O.candidate_pairs(m.x, m.tri)
    ev = O.evaluate(m.x, m.tri, pairs)
    assert E == pytest.approx(float(ev.T.sum()), rel=1e-14)        # springs at rest add nothing
    g0, blocks = O.assemble(m.tri, ev, m.V)
    assert np.array_equal(grad, g0)
    assert len(rows) == m.V                                          # every vertex has a spring
    for key, b in O.elastic_blocks(m.x, el).items():
        blocks[key] = blocks[key] + b if key in blocks else b
    H = O.blocks_to_dense(blocks, rows)
    mu = prm.mu_rel * np.mean(np.diag(H))
    r = (H + mu * np.eye(len(H))) @ d[rows].ravel() + grad[rows].ravel()
    assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(grad)
    assert np.sum(grad * d) < 0


def test_elastic_system_composition():
    """The Newton system of E_el + sum T (prestressed springs and anchors, so the elastic part
    is not zero): its energy is the pairs' sum T plus the elastic energy, and its gradient minus
    the pairs' assembled gradient is the derivative of the elastic energy, checked by central
    differences (the elastic term is smooth; T jumps where a vertex crosses a face, so the
    total is not differenced)."""
    m = ti.cloth(12, seed=21)
    rng = np.random.default_rng(7)
    e = O.mesh_edges(m.tri)
    rest = rng.uniform(0.8, 1.2, len(e)) * np.linalg.norm(m.x[e[:, 0]] - m.x[e[:, 1]], axis=1)
    anchors = np.array([3, 50, 100])
    el = O.Elastic(e, rest, 0.5, anchors, m.x[anchors] + 0.02, 2.0)
    prm = O.NewtonParams()
    E, n, grad, _, _ = O.newton_direction_elastic(m.x, m.tri, None, prm, el)
    assert n > 0
    sum_T = O.energy(m.x, m.tri, None, prm)[0]
    E_el = O.elastic_energy(m.x, el)
    assert E_el > 1e-2 * sum_T
    assert E == pytest.approx(sum_T + E_el, rel=1e-13)
    assert O.total_energy(m.x, m.tri, None, prm, el)[0] == pytest.approx(sum_T + E_el, rel=1e-13)
    ev = O.evaluate(m.x, m.tri, O.candidate_pairs(m.x, m.tri))
    g_el = grad - O.assemble(m.tri, ev, m.V)[0]
    h = 1e-6
    for _ in range(4):
        v = rng.standard_normal(m.x.shape)
        fd = (O.elastic_energy(m.x + h * v, el) - O.elastic_energy(m.x - h * v, el)) / (2 * h)
        assert fd == pytest.approx(float(np.sum(g_el * v)), rel=1e-6)


def test_zero_length_spring():
    """A spring whose ends coincide has no direction: its gradient is 0 and its Hessian block the
    limit k I of the stretched case along any direction (the energy is k/2 L^2 there)."""
    k, L = 2.0, 0.3
    x = np.array([[0.5, -0.2, 1.0], [0.5, -0.2, 1.0]])
    el = O.Elastic(np.array([[0, 1]]), np.array([L]), k)
    assert O.elastic_energy(x, el) == pytest.approx(0.5 * k * L * L, rel=1e-14)
    assert not O.elastic_gradient(x, el).any()
    H = O.spring_hessian(x[0], x[1], L, k)
    assert np.array_equal(H[:3, :3], k * np.eye(3)) and np.array_equal(H[:3, 3:], -k * np.eye(3))
