"""Batched independent instances (intra-group pair mode): one Newton step solves every group
on its own.  Checked against the oracle (each group's direction is the solution of its own
regularised system, scaled by its own step cap) and against stepping each group alone with
the single-problem path (same accepted step, same positions up to the solvers' rounding)."""
import numpy as np
import pytest
import torch

import oracle as O
import ttie_inputs as ti

pytestmark = pytest.mark.gpu

MODE_INTRA = 2


@pytest.fixture(scope="module")
def ttie():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06511_gb300 import ttie as t
    return t


@pytest.fixture(scope="module")
def batch():
    m, vo, to = ti.ellipsoid_batch(8, seed=4, f_min=60, f_max=700)
    return m, vo, to


def _dev(m, dt):
    return (torch.tensor(m.x, dtype=dt, device="cuda"), torch.tensor(m.tri, dtype=torch.int32, device="cuda"),
            torch.tensor(m.group, dtype=torch.int32, device="cuda"))


def _instance(m, vo, to, k):
    x = m.x[vo[k]:vo[k + 1]]
    tri = m.tri[to[k]:to[k + 1]] - vo[k]
    return ti.Mesh(x.copy(), tri.astype(np.int32), np.zeros(len(tri), np.int32))


@pytest.mark.parametrize("precond", ["auto", "block_jacobi", "chebyshev"])
def test_batched_direction_is_each_instance_solution(ttie, batch, precond):
    """Each instance's direction against a dense solve of its own oracle system, with each
    preconditioner of the batched PCG (AUTO: Chebyshev for instances in shared memory)."""
    m, vo, to = batch
    x, tri, grp = _dev(m, torch.float64)
    pc = {"auto": ttie.PCG_AUTO, "block_jacobi": ttie.PCG_BLOCK_JACOBI, "chebyshev": ttie.PCG_CHEBYSHEV}[precond]
    prm = dict(precision=ttie.F64, pair_mode=MODE_INTRA, pcg_rtol=1e-9, pcg_max_it=4000, max_step=1.0,
               pcg_precond=pc)
    ctx = ttie.Context(**prm)
    ctx.build_bvh(x, tri, grp)
    info = ctx.newton_step(x.clone())
    assert info["n_active"] > 0
    d = ctx.get_direction().cpu().numpy()
    checked = 0
    for k in range(len(vo) - 1):
        mk = _instance(m, vo, to, k)
        pairs = O.candidate_pairs(mk.x, mk.tri)
        ev = O.evaluate(mk.x, mk.tri, pairs)
        dk = d[vo[k]:vo[k + 1]]
        if not ev.active.any():
            assert np.all(dk == 0)
            continue
        g, blocks = O.assemble(mk.tri, ev, mk.V)
        verts = np.array(sorted({r for (r, c) in blocks}))
        H = O.blocks_to_dense(blocks, verts)
        mu = 1e-3 * np.trace(H) / len(H)
        sol = np.linalg.solve(H + mu * np.eye(len(H)), -g[verts].ravel()).reshape(-1, 3)
        e = mk.x[mk.tri[:, [1, 2, 0]]] - mk.x[mk.tri]
        cap = 1.0 * np.linalg.norm(e, axis=-1).mean()
        dmax = np.linalg.norm(sol, axis=1).max()
        want = np.zeros_like(dk)
        want[verts] = sol * (cap / dmax if dmax > cap else 1.0)
        assert np.abs(dk - want).max() <= 1e-6 * np.abs(want).max(), k
        checked += 1
    assert checked >= 3


def test_batched_step_matches_each_instance_alone(ttie, batch):
    m, vo, to = batch
    x, tri, grp = _dev(m, torch.float64)
    prm = dict(precision=ttie.F64, pcg_rtol=1e-9, pcg_max_it=4000)
    ctx = ttie.Context(pair_mode=MODE_INTRA, **prm)
    ctx.build_bvh(x, tri, grp)
    xb = x.clone()
    ctx.newton_step(xb)
    xb = xb.cpu().numpy()
    x0 = m.x
    moved = 0
    for k in range(len(vo) - 1):
        mk = _instance(m, vo, to, k)
        xs, ts, _ = _dev(mk, torch.float64)
        c1 = ttie.Context(pair_mode=0, **prm)
        c1.build_bvh(xs, ts)
        inf = c1.newton_step(xs)
        step_alone = xs.cpu().numpy() - mk.x
        step_batch = xb[vo[k]:vo[k + 1]] - x0[vo[k]:vo[k + 1]]
        scale = max(np.abs(step_alone).max(), 1e-300)
        assert np.abs(step_batch - step_alone).max() <= 1e-6 * scale, (k, inf["alpha"])
        moved += inf["n_active"] > 0
    assert moved >= 3


def test_batched_solve_energy_falls(ttie, batch):
    m, vo, to = batch
    x, tri, grp = _dev(m, torch.float32)
    ctx = ttie.Context(pair_mode=MODE_INTRA)
    ctx.build_bvh(x, tri, grp)
    E0, n0 = ctx.eval_pairs(x, ttie.EVAL_E)
    for _ in range(5):
        inf = ctx.newton_step(x)
        assert np.isfinite(inf["energy_new"]) and inf["grad_dot_dir"] < 0
    E1, n1 = ctx.eval_pairs(x, ttie.EVAL_E)
    assert E1 < 0.5 * E0


def test_batched_layout_errors(ttie, batch):
    m, vo, to = batch
    # a vertex used by two groups
    bad = ti.Mesh(m.x.copy(), m.tri.copy(), m.group.copy())
    bad.tri[to[1]] = [bad.tri[0, 0], bad.tri[to[1], 1], bad.tri[to[1], 2]]
    x, tri, grp = _dev(bad, torch.float32)
    ctx = ttie.Context(pair_mode=MODE_INTRA)
    with pytest.raises(ttie.TTIEError) as e:
        ctx.build_bvh(x, tri, grp)
    assert e.value.status == ttie.TTIE_ERR_INVALID
    # vertices of the groups interleaved: the instances' rows are not contiguous
    rng = np.random.default_rng(0)
    perm = rng.permutation(m.V)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(m.V)
    shuf = ti.Mesh(m.x[perm].copy(), inv[m.tri].astype(np.int32), m.group.copy())
    x, tri, grp = _dev(shuf, torch.float32)
    ctx = ttie.Context(pair_mode=MODE_INTRA)
    ctx.build_bvh(x, tri, grp)
    with pytest.raises(ttie.TTIEError) as e:
        ctx.newton_step(x)
    assert e.value.status == ttie.TTIE_ERR_INVALID


def test_batched_block_size_does_not_change_results(ttie, batch):
    """Every reduction of the per-instance PCG runs in an order fixed by the instance alone, so
    the block size the tuner picks changes the speed, not a bit of the result."""
    m, vo, to = batch
    outs = []
    for t in (128, 512, 1024, 0):
        x, tri, grp = _dev(m, torch.float32)
        ctx = ttie.Context(pair_mode=MODE_INTRA, inst_threads=t)
        ctx.build_bvh(x, tri, grp)
        for _ in range(2):
            ctx.newton_step(x)
        outs.append(x.cpu())
    for o in outs[1:]:
        assert torch.equal(o, outs[0])


@pytest.mark.parametrize("precond", ["auto", "chebyshev"])
def test_batched_large_instances_in_global_memory(ttie, precond):
    """Instances too large for one block's shared memory keep their PCG vectors and matrix rows
    in global memory (block Jacobi under AUTO; the Chebyshev polynomial's vectors in global
    memory too when asked for); the step still equals stepping each instance alone."""
    m, vo, to = ti.ellipsoid_batch(2, seed=7, f_min=12000, f_max=16000)
    x, tri, grp = _dev(m, torch.float64)
    prm = dict(precision=ttie.F64, pcg_rtol=1e-9, pcg_max_it=4000)
    ctx = ttie.Context(pair_mode=MODE_INTRA, pcg_precond=ttie.PCG_AUTO if precond == "auto" else ttie.PCG_CHEBYSHEV,
                       **prm)
    ctx.build_bvh(x, tri, grp)
    info = ctx.newton_step(x)
    # FP64: 244 B per row and 76 B per 3x3 block; an instance needs more than a block's 220 KB
    assert (info["n_rows"] * 244 + info["nnzb"] * 76) / 2 > 220 * 1024
    xb = x.cpu().numpy()
    for k in range(2):
        mk = _instance(m, vo, to, k)
        xs, ts, _ = _dev(mk, torch.float64)
        c1 = ttie.Context(pair_mode=0, **prm)
        c1.build_bvh(xs, ts)
        c1.newton_step(xs)
        step_alone = xs.cpu().numpy() - mk.x
        step_batch = xb[vo[k]:vo[k + 1]] - m.x[vo[k]:vo[k + 1]]
        scale = max(np.abs(step_alone).max(), 1e-300)
        assert np.abs(step_batch - step_alone).max() <= 1e-6 * scale, k
