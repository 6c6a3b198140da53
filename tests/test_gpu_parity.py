"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results are compared bit-exactly: the candidate pair set (closed box
overlap, non-adjacent), the intersecting pair set and the block pattern.  Values
meet the stated tolerances in both forms (FP32 positions and FP64): T relative
1e-5, gradients and Hessian blocks relative 1e-4, on pairs with
min(|t_c^0|, |t_c^1|) > 1e-6 of the bounding-box diagonal (``_cases``).
"""
import numpy as np
import pytest
import torch

import oracle as O
import ttie_inputs as ti
from _cases import (G_RTOL, H_RTOL, MODE, T_RTOL, block_errors, pair_errors, pair_set, small_cases,
                    tolerance_mask)

pytestmark = pytest.mark.gpu

CASES = small_cases()


@pytest.fixture(scope="module")
def ttie():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06511_gb300 import ttie as t
    return t


def _ctx(ttie, mode, precision=0, brute=False, **kw):
    pm = MODE[mode] | (ttie.PAIRS_BRUTE if brute else 0)
    return ttie.Context(precision=precision, pair_mode=pm, **kw)


def _dev(m, dtype=torch.float32):
    x = torch.tensor(m.x, dtype=dtype, device="cuda")
    tri = torch.tensor(m.tri, dtype=torch.int32, device="cuda")
    grp = torch.tensor(m.group, dtype=torch.int32, device="cuda")
    return x, tri, grp


_oracle_cache = {}


def _oracle(name):
    if name not in _oracle_cache:
        m, mode = CASES[name]
        pairs = O.candidate_pairs(m.x, m.tri, m.group, mode)
        ev = O.evaluate(m.x, m.tri, pairs)
        _oracle_cache[name] = (pairs, ev)
    return _oracle_cache[name]


@pytest.mark.parametrize("name", list(CASES))
def test_candidates_bit_exact(ttie, name):
    m, mode = CASES[name]
    x, tri, grp = _dev(m)
    ctx = _ctx(ttie, mode)
    n = ctx.build_bvh(x, tri, grp)
    got = ctx.get_candidates().cpu().numpy()
    pairs, _ = _oracle(name)
    assert n == len(pairs)
    assert np.all(got[:, 0] < got[:, 1])
    assert pair_set(got) == pair_set(pairs)
    # deterministic order
    ctx.build_bvh(x, tri, grp)
    assert np.array_equal(ctx.get_candidates().cpu().numpy(), got)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("exact_only", [0, 1, 2])
def test_active_set_bit_exact(ttie, name, exact_only):
    """Intersecting pairs bit-exact against the oracle's exact test: with the filters (0), every
    sign exact (1: float32 points in 256-bit integers where their span fits, else expansions),
    every sign by expansion arithmetic (2)."""
    m, mode = CASES[name]
    x, tri, grp = _dev(m)
    ctx = _ctx(ttie, mode, exact_only=exact_only)
    ctx.build_bvh(x, tri, grp)
    E, n_act = ctx.eval_pairs(x, ttie.EVAL_E)
    pairs, ev = _oracle(name)
    act_pairs, _, _ = ctx.get_active(with_derivatives=False)
    assert n_act == int(ev.active.sum())
    assert pair_set(act_pairs.cpu().numpy()) == pair_set(pairs[ev.active])
    st = ctx.get_filter_stats()
    if exact_only:
        assert st["fp32"] == 0 and st["fp64"] == 0


def test_exact_zeros_settled_before_expansions(ttie):
    """Mirror-symmetric lat-long ellipsoids (the second with equal x and y semi-axes, so vertex
    quadruples symmetric about x = 0, y = 0 and x = y are exactly coplanar; coordinates below
    1e-6 set to 0): every orientation sign neither filter certifies is an exact zero or a
    determinant whose entries fit the 128-bit integer evaluation, so none reaches the expansion
    arithmetic, and the intersecting set equals the exact oracle's."""
    from ttie_inputs.meshes import Mesh, concat
    m1 = ti.ellipsoid(14, (1.0, 0.8, 0.6))
    m2 = ti.ellipsoid(10, (0.7, 0.7, 0.9))
    m = concat([m1, Mesh(m2.x + np.array([0.0, 0.0, 0.5]), m2.tri, m2.group)]).as_f32()
    m.x[np.abs(m.x) < 1e-6] = 0.0
    x, tri, grp = _dev(m)
    ctx = _ctx(ttie, "self")
    ctx.build_bvh(x, tri, grp)
    E, n_act = ctx.eval_pairs(x, ttie.EVAL_E)
    pairs = O.candidate_pairs(m.x, m.tri, m.group, "self")
    ev = O.evaluate(m.x, m.tri, pairs)
    act_pairs, _, _ = ctx.get_active(with_derivatives=False)
    assert n_act == int(ev.active.sum()) > 0
    assert pair_set(act_pairs.cpu().numpy()) == pair_set(pairs[ev.active])
    st = ctx.get_filter_stats()
    assert st["fp64"] > 0 and st["exact"] == 0, st


@pytest.mark.parametrize("exact_only", [0, 1, 2])
def test_wide_coordinate_span_bit_exact(ttie, exact_only):
    """Triangles whose coordinates span about 60 binary orders (1e-17 next to 1: the lat-long
    vertices at cos(pi/2) and sin(pi), not snapped), coplanar and crossing by construction:
    signs whose integer evaluation needs the 256-bit path, and exact zeros among them.  The
    intersecting set equals the exact oracle's with the filters, with every sign exact, and with
    expansion arithmetic only."""
    from ttie_inputs.meshes import Mesh, concat
    m1 = ti.ellipsoid(12, (1.0, 0.8, 0.6))
    m2 = ti.ellipsoid(8, (0.7, 0.7, 0.9))
    m = concat([m1, Mesh(m2.x + np.array([0.0, 0.0, 0.5]), m2.tri, m2.group)]).as_f32()
    tiny = np.abs(m.x[m.x != 0]).min()
    assert tiny < 1e-15   # the span the 128-bit evaluation cannot hold
    x, tri, grp = _dev(m)
    ctx = _ctx(ttie, "self", exact_only=exact_only)
    ctx.build_bvh(x, tri, grp)
    E, n_act = ctx.eval_pairs(x, ttie.EVAL_E)
    pairs = O.candidate_pairs(m.x, m.tri, m.group, "self")
    ev = O.evaluate(m.x, m.tri, pairs)
    act_pairs, _, _ = ctx.get_active(with_derivatives=False)
    assert n_act == int(ev.active.sum()) > 0
    assert pair_set(act_pairs.cpu().numpy()) == pair_set(pairs[ev.active])


def _match(ctx, pairs, ev):
    ap, tc, dtc = ctx.get_active()
    ap = ap.cpu().numpy().astype(np.int64)
    tc = tc.double().cpu().numpy()
    dtc = dtc.double().cpu().numpy()
    idx = {tuple(p): k for k, p in enumerate(pairs.tolist())}
    k = np.array([idx[tuple(p)] for p in ap.tolist()], dtype=np.int64)
    return ap, tc, dtc, k


def _pair_size(m, pairs):
    v = np.concatenate([m.x[m.tri[pairs[:, 0]]], m.x[m.tri[pairs[:, 1]]]], axis=1)
    return (v.max(1) - v.min(1)).max(1)


@pytest.mark.parametrize("name", ["cloth40", "spheres_inter", "soup", "tori", "ellipsoids_intra", "snapped_grid"])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_pair_values_meet_stated_tolerances(ttie, name, prec):
    """T, the Eq. 3 gradient and the projected Eq. 4 Hessian of every intersecting pair in the
    tolerance mask, per pair, against the oracle.  On the snapped grid many pairs sit exactly at
    a tie of the construction (an interval end point shared, a cut vertex on the plane), where
    t_c is not differentiable and either one-sided gradient is correct: there only T and the
    energy are compared."""
    m, mode = CASES[name]
    precision = ttie.F64 if prec == "f64" else ttie.F32
    x, tri, grp = _dev(m, torch.float64 if prec == "f64" else torch.float32)
    ctx = _ctx(ttie, mode, precision=precision)
    ctx.build_bvh(x, tri, grp)
    E, n_act = ctx.eval_pairs(x, ttie.EVAL_E | ttie.EVAL_H)
    pairs, ev = _oracle(name)
    ap, tc, dtc, k = _match(ctx, pairs, ev)
    sub = O.PairEval(ev.pairs[k], ev.tc[k], ev.dtc[k], ev.sides64[k], ev.flags64[k], ev.active[k])
    mask = tolerance_mask(m.x, sub.tc)
    assert mask.mean() > 0.9
    eT, eg, eH = pair_errors(tc, dtc, sub)
    assert eT[mask].max() <= T_RTOL, eT[mask].max()
    assert abs(E - ev.T.sum()) <= T_RTOL * ev.T.sum()
    if name == "snapped_grid":
        return
    assert eg[mask].max() <= G_RTOL, (eg[mask].max(), ap[mask][np.argmax(eg[mask])])
    assert eH[mask].max() <= H_RTOL, (eH[mask].max(), ap[mask][np.argmax(eH[mask])])


@pytest.mark.parametrize("name", ["spheres_inter", "cloth40"])
def test_fp64_form_meets_relative_tolerances(ttie, name):
    m, mode = CASES[name]
    x, tri, grp = _dev(m, torch.float64)
    ctx = _ctx(ttie, mode, precision=ttie.F64, brute=(name == "spheres_inter"))
    n = ctx.build_bvh(x, tri, grp)
    if name == "spheres_inter":
        assert n == 320 * 320
    E, n_act = ctx.eval_pairs(x, ttie.EVAL_E | ttie.EVAL_H)
    pairs, ev = _oracle(name)
    assert n_act == int(ev.active.sum())
    ap, tc, dtc, k = _match(ctx, pairs, ev)
    sub = O.PairEval(ev.pairs[k], ev.tc[k], ev.dtc[k], ev.sides64[k], ev.flags64[k], ev.active[k])
    mask = tolerance_mask(m.x, sub.tc)
    eT, eg, eH = pair_errors(tc, dtc, sub)
    assert eT[mask].max() <= T_RTOL and eg[mask].max() <= G_RTOL and eH[mask].max() <= H_RTOL
    assert E == pytest.approx(ev.T.sum(), rel=1e-9)


@pytest.mark.parametrize("name,precision", [("cloth40", 0), ("tori", 0), ("spheres_inter", 1)])
def test_assembly_pattern_and_values(ttie, name, precision):
    m, mode = CASES[name]
    dt = torch.float64 if precision else torch.float32
    x, tri, grp = _dev(m, dt)
    ctx = _ctx(ttie, mode, precision=precision)
    ctx.build_bvh(x, tri, grp)
    grad_full = torch.zeros((m.V, 3), dtype=dt, device="cuda")
    ctx.eval_pairs(x, ttie.EVAL_E | ttie.EVAL_G | ttie.EVAL_H, grad=grad_full)
    bsr = ctx.assemble()
    pairs, ev = _oracle(name)
    grad_or, blocks = O.assemble(m.tri, ev, m.V)
    rows = bsr.vertex_of_row.cpu().numpy()
    rp = bsr.row_ptr.cpu().numpy()
    ci = bsr.col_idx.cpu().numpy()
    val = bsr.val.double().cpu().numpy()
    got = {}
    for r in range(len(rows)):
        for b in range(rp[r], rp[r + 1]):
            got[(int(rows[r]), int(rows[ci[b]]))] = val[b]
    assert set(got) == set(blocks)                      # pattern bit-exact
    assert np.all(np.diff(rows) > 0)
    for r in range(len(rows)):                          # columns ascending within a row
        assert np.all(np.diff(ci[rp[r]:rp[r + 1]]) > 0)
    # blocks relative to sqrt(|H_rr| |H_cc|); gradient rows relative to the sum of the sizes
    # of the pair gradients they add up (the stated 1e-4 in both forms)
    eb = block_errors(got, blocks)
    assert eb.max() <= H_RTOL, eb.max()
    vid = O.pair_dofs(m.tri, ev.pairs[ev.active])
    gp = np.abs(O.gradient(ev)[ev.active])
    contrib = np.zeros((m.V, 3))
    for r in range(6):
        np.add.at(contrib, vid[:, r], gp[:, 3 * r:3 * r + 3])
    scale = contrib.max(1, keepdims=True)
    g = grad_full.double().cpu().numpy()
    assert (np.abs(g - grad_or) <= G_RTOL * scale).all()
    assert (np.abs(bsr.grad.double().cpu().numpy() - grad_or[rows]) <= G_RTOL * scale[rows]).all()
    # deterministic
    ctx.eval_pairs(x, ttie.EVAL_E | ttie.EVAL_H)
    bsr2 = ctx.assemble()
    assert torch.equal(bsr2.val, bsr.val) and torch.equal(bsr2.col_idx, bsr.col_idx)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("precond", ["block_jacobi", "auto", "streamed", "uncached", "uncached_auto"])
def test_pcg_matches_direct_solve(ttie, precision, precond):
    """The PCG's solution against a dense direct solve of the same system (the matrix the GPU
    assembled, read back in FP64): the true residual is at the requested level and the
    solution error is below a fixed bound (FP32 2e-3, FP64 1e-6).  The residual on the
    oracle's own matrix adds the assembly's rounding.  Kernels: the block-resident one with
    its matrix rows in shared memory (block Jacobi; AUTO, which picks Chebyshev here) or read
    from global memory on every product (the product of systems too large for shared memory:
    "uncached", both preconditioners), and the streamed kernels."""
    name = "cloth40"
    m, mode = CASES[name]
    dt = torch.float64 if precision else torch.float32
    x, tri, grp = _dev(m, dt)
    kernel = {"streamed": ttie.PCG_KERNEL_STREAMED, "uncached": ttie.PCG_KERNEL_RESIDENT_UNCACHED,
              "uncached_auto": ttie.PCG_KERNEL_RESIDENT_UNCACHED}.get(precond, ttie.PCG_KERNEL_RESIDENT)
    ctx = _ctx(ttie, mode, precision=precision,
               pcg_precond=ttie.PCG_AUTO if precond in ("auto", "uncached_auto") else ttie.PCG_BLOCK_JACOBI,
               pcg_kernel=kernel)
    ctx.build_bvh(x, tri, grp)
    ctx.eval_pairs(x, ttie.EVAL_E | ttie.EVAL_H)
    bsr = ctx.assemble()
    rhs = -bsr.grad
    rtol = 1e-9 if precision else 1e-5
    d, iters, rel = ctx.pcg(rhs.contiguous(), rtol=rtol, max_it=5000)
    assert rel <= rtol
    rows = bsr.vertex_of_row.cpu().numpy()
    rp = bsr.row_ptr.cpu().numpy()
    ci = bsr.col_idx.cpu().numpy()
    val = bsr.val.double().cpu().numpy().reshape(-1, 3, 3)
    n = len(rows)
    Hg = np.zeros((3 * n, 3 * n))
    for r in range(n):
        for b in range(rp[r], rp[r + 1]):
            Hg[3 * r:3 * r + 3, 3 * ci[b]:3 * ci[b] + 3] = val[b]
    mu = 1e-3 * np.mean(np.diag(Hg))
    A = Hg + mu * np.eye(3 * n)
    b = -bsr.grad.double().cpu().numpy().ravel()
    sol = np.linalg.solve(A, b)
    dd = d.double().cpu().numpy().ravel()
    res = np.linalg.norm(A @ dd - b) / np.linalg.norm(b)
    assert res <= (2 * rtol if precision else 5 * rtol), (res, iters, rel)
    err = np.linalg.norm(dd - sol) / np.linalg.norm(sol)
    assert err <= (1e-6 if precision else 2e-3), (err, res, iters)
    pairs, ev = _oracle(name)
    _, blocks = O.assemble(m.tri, ev, m.V)
    Ho = O.blocks_to_dense(blocks, rows)
    Ao = Ho + 1e-3 * np.mean(np.diag(Ho)) * np.eye(len(Ho))
    res_o = np.linalg.norm(Ao @ dd - b) / np.linalg.norm(b)
    assert res_o <= (1e-8 if precision else 1e-3), res_o


def test_newton_step_descends(ttie):
    m, mode = CASES["cloth40"]
    x, tri, grp = _dev(m)
    ctx = _ctx(ttie, mode)
    ctx.build_bvh(x, tri, grp)
    info = ctx.newton_step(x)
    assert info["n_active"] > 0 and info["grad_dot_dir"] < 0
    assert info["energy_new"] < info["energy"] or info["n_active_new"] == 0
    assert info["n_candidates_swept"] >= info["n_candidates"]
    d = ctx.get_direction()
    assert torch.isfinite(d).all()


@pytest.mark.parametrize("case", ["spheres_shallow", "cloth_mild"])
def test_solve_certified_intersection_free(ttie, case):
    if case == "spheres_shallow":
        m, mode = ti.two_icospheres(offset=(1.95, 0.0, 0.0)).as_f32(), "inter"
    else:
        m, mode = ti.cloth(16, seed=2, shear=0.05).as_f32(), "self"
    x, tri, grp = _dev(m)
    ctx = _ctx(ttie, mode, newton_max_it=40)
    ctx.build_bvh(x, tri, grp)
    info = ctx.solve(x)
    assert info["converged"] == 1, info
    xf = x.double().cpu().numpy()
    assert O.certify(xf, m.tri, m.group, mode) == 0


def test_errors_are_status_codes(ttie):
    m, mode = CASES["cloth40"]
    x, tri, grp = _dev(m)
    ctx = _ctx(ttie, mode)
    with pytest.raises(ttie.TTIEError) as e:
        ctx.eval_pairs(x)
    assert e.value.status == ttie.TTIE_ERR_STATE
    bad = tri.clone()
    bad[5, 1] = m.V + 3
    with pytest.raises(ttie.TTIEError) as e:
        ctx.build_bvh(x, bad)
    assert e.value.status == ttie.TTIE_ERR_INVALID
    xn = x.clone()
    xn[7, 2] = float("nan")
    with pytest.raises(ttie.TTIEError) as e:
        ctx.build_bvh(xn, tri)
    assert e.value.status == ttie.TTIE_ERR_NONFINITE
    ctx.build_bvh(x, tri)
    with pytest.raises(ttie.TTIEError) as e:
        ctx.eval_pairs(xn)
    assert e.value.status == ttie.TTIE_ERR_NONFINITE
    # the context stays usable after errors
    ctx.build_bvh(x, tri)
    E, n = ctx.eval_pairs(x)
    assert n > 0


def test_degenerate_sizes(ttie):
    ctx = _ctx(ttie, "self")
    x = torch.tensor([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=torch.float32, device="cuda")
    tri = torch.tensor([[0, 1, 2]], dtype=torch.int32, device="cuda")
    assert ctx.build_bvh(x, tri) == 0
    assert ctx.eval_pairs(x) == (0.0, 0)
    assert ctx.newton_step(x)["n_active"] == 0
    tri0 = torch.zeros((0, 3), dtype=torch.int32, device="cuda")
    assert ctx.build_bvh(x, tri0) == 0
    assert ctx.eval_pairs(x) == (0.0, 0)


@pytest.mark.parametrize("name", ["cloth40", "tori", "soup"])
@pytest.mark.parametrize("psd", ["drop_cross", "whole"])
def test_assembly_psd_modes(ttie, name, psd):
    """The other projections of §1.1 against the oracle: parts 1 and 2 only, and the eigenvalue
    clamp of the whole Eq. 4 Hessian (numpy eigh of the 18x18 sum in the oracle, a 2x2
    reduction on the GPU)."""
    m, mode = CASES[name]
    x, tri, grp = _dev(m, torch.float64)
    mode_id = {"drop_cross": ttie.PSD_DROP_CROSS, "whole": ttie.PSD_WHOLE}[psd]
    ctx = _ctx(ttie, mode, precision=1, psd_mode=mode_id)
    ctx.build_bvh(x, tri, grp)
    ctx.eval_pairs(x, ttie.EVAL_E | ttie.EVAL_H)
    bsr = ctx.assemble()
    pairs, ev = _oracle(name)
    _, blocks = O.assemble(m.tri, ev, m.V, psd=psd)
    rows = bsr.vertex_of_row.cpu().numpy()
    rp = bsr.row_ptr.cpu().numpy()
    ci = bsr.col_idx.cpu().numpy()
    val = bsr.val.cpu().numpy()
    got = {}
    for r in range(len(rows)):
        for b in range(rp[r], rp[r + 1]):
            got[(int(rows[r]), int(rows[ci[b]]))] = val[b]
    assert set(got) == set(blocks)
    scale = max(np.abs(b).max() for b in blocks.values())
    for key, b in blocks.items():
        assert np.allclose(got[key], b, rtol=1e-4, atol=1e-4 * scale), key


@pytest.mark.parametrize("name", list(CASES))
def test_hash_candidates_bit_exact(ttie, name):
    """The spatial-hashing broad phase (TTIE_PAIRS_HASH) gives the oracle's candidate set in
    every pair mode, in a deterministic order, and the same evaluation as the LBVH's list."""
    m, mode = CASES[name]
    x, tri, grp = _dev(m)
    ctx = ttie.Context(pair_mode=MODE[mode] | ttie.PAIRS_HASH)
    n = ctx.build_bvh(x, tri, grp)
    got = ctx.get_candidates().cpu().numpy()
    pairs, ev = _oracle(name)
    assert n == len(pairs)
    assert np.all(got[:, 0] < got[:, 1])
    assert pair_set(got) == pair_set(pairs)
    ctx.build_bvh(x, tri, grp)
    assert np.array_equal(ctx.get_candidates().cpu().numpy(), got)
    E, n_act = ctx.eval_pairs(x, ttie.EVAL_E)
    assert n_act == int(ev.active.sum())
    assert E == pytest.approx(float(ev.T.sum()), rel=1e-5, abs=1e-30)


def test_hash_candidates_match_lbvh_full_size(ttie):
    m = ti.cloth(256, seed=2).as_f32()
    x, tri, grp = _dev(m)
    sets = []
    for flag in (0, ttie.PAIRS_HASH):
        ctx = ttie.Context(pair_mode=flag)
        ctx.build_bvh(x, tri)
        c = ctx.get_candidates().cpu().numpy().astype(np.int64)
        sets.append(np.sort(c[:, 0] * m.F + c[:, 1]))
    assert len(sets[0]) > 600000 and np.array_equal(sets[0], sets[1])


def test_pcg_wait_runs_out_and_context_stays_usable(ttie):
    """Failure path of the block-resident PCG, without a GPU fault: with the test switch set,
    block 0 never publishes its partial sums, every block's wait for them runs out after about a
    second (a bound on elapsed time), the kernel returns and the call reports TTIE_ERR_CUDA; the
    same context then solves the same system normally."""
    import time
    m, mode = CASES["cloth40"]
    x, tri, grp = _dev(m)
    ctx = _ctx(ttie, mode)
    ctx.build_bvh(x, tri, grp)
    ctx.eval_pairs(x, ttie.EVAL_E | ttie.EVAL_H)
    bsr = ctx.assemble()
    rhs = (-bsr.grad).contiguous()
    ctx.set_params(test_withhold=1)
    t0 = time.time()
    with pytest.raises(ttie.TTIEError) as e:
        ctx.pcg(rhs, rtol=1e-6, max_it=50)
    assert e.value.status == ttie.TTIE_ERR_CUDA
    assert time.time() - t0 < 20.0
    ctx.set_params(test_withhold=0)
    d, iters, rel = ctx.pcg(rhs, rtol=1e-4, max_it=5000)
    assert rel <= 1e-4 and torch.isfinite(d).all()
