"""The alternative kernels of two stages against each other, on the same inputs.

* LBVH traversal: the one-walk traversal (the default) gives the same candidate list in the
  same order as the two-walk traversal, so every later result is identical.
* Chebyshev-preconditioned PCG (TTIE_PCG_CHEBYSHEV, what TTIE_PCG_AUTO picks for systems
  whose matrix rows fit shared memory): the same bar as the block-Jacobi PCG (residual at the
  requested level on the system it solved, fixed bound on the solution error against a dense
  direct solve).
"""
import numpy as np
import pytest
import torch

import ttie_inputs as ti
from _cases import MODE, small_cases

pytestmark = pytest.mark.gpu

CASES = small_cases()


@pytest.fixture(scope="module")
def ttie():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06511_gb300 import ttie as t
    return t


def _dev(m, dtype=torch.float32):
    return (torch.tensor(m.x, dtype=dtype, device="cuda"), torch.tensor(m.tri, dtype=torch.int32, device="cuda"),
            torch.tensor(m.group, dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("name", list(CASES))
def test_one_walk_traversal_same_list(ttie, name):
    m, mode = CASES[name]
    x, tri, grp = _dev(m)
    out = []
    for tm in (ttie.TRAVERSAL_TWO_WALKS, ttie.TRAVERSAL_ONE_WALK):
        ctx = ttie.Context(pair_mode=MODE[mode], traversal_mode=tm)
        n = ctx.build_bvh(x, tri, grp)
        E, n_act = ctx.eval_pairs(x, ttie.EVAL_E)
        out.append((n, ctx.get_candidates().cpu(), E, n_act))
    assert out[0][0] == out[1][0]
    assert torch.equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2] and out[0][3] == out[1][3]


def test_one_walk_traversal_newton_steps_identical(ttie):
    """Full size, several Newton steps (line-search sweeps over refitted trees included): the
    two traversals give bit-identical iterates."""
    m = ti.cloth(256, seed=2).as_f32()
    x0, tri, _ = _dev(m)
    res = []
    for tm in (ttie.TRAVERSAL_TWO_WALKS, ttie.TRAVERSAL_ONE_WALK):
        x = x0.clone()
        ctx = ttie.Context(traversal_mode=tm)
        ctx.build_bvh(x, tri)
        infos = [ctx.newton_step(x) for _ in range(3)]
        res.append((x, [(i["n_candidates"], i["n_candidates_swept"], i["n_active"], i["energy_new"]) for i in infos]))
    assert res[0][1] == res[1][1]
    assert torch.equal(res[0][0], res[1][0])


def _dense(bsr):
    rp = bsr.row_ptr.cpu().numpy()
    ci = bsr.col_idx.cpu().numpy()
    val = bsr.val.double().cpu().numpy()
    n = len(rp) - 1
    H = np.zeros((3 * n, 3 * n))
    for r in range(n):
        for b in range(rp[r], rp[r + 1]):
            H[3 * r:3 * r + 3, 3 * ci[b]:3 * ci[b] + 3] = val[b]
    return H


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("degree", [2, 3])
def test_chebyshev_pcg_matches_direct_solve(ttie, precision, degree):
    m, mode = CASES["cloth40"]
    dt = torch.float64 if precision else torch.float32
    x, tri, grp = _dev(m, dt)
    ctx = ttie.Context(precision=precision, pcg_precond=ttie.PCG_CHEBYSHEV, pcg_cheb_degree=degree)
    ctx.build_bvh(x, tri, grp)
    ctx.eval_pairs(x, ttie.EVAL_E | ttie.EVAL_H)
    bsr = ctx.assemble()
    rhs = (-bsr.grad).contiguous()
    rtol = 1e-9 if precision else 1e-5
    d, iters, rel = ctx.pcg(rhs, rtol=rtol, max_it=5000)
    assert rel <= rtol and iters > 6
    H = _dense(bsr)
    A = H + 1e-3 * np.mean(np.diag(H)) * np.eye(len(H))
    b = rhs.double().cpu().numpy().ravel()
    dd = d.double().cpu().numpy().ravel()
    res = np.linalg.norm(A @ dd - b) / np.linalg.norm(b)
    assert res <= (2 * rtol if precision else 5 * rtol), (res, iters, rel)
    sol = np.linalg.solve(A, b)
    err = np.linalg.norm(dd - sol) / np.linalg.norm(sol)
    assert err <= (1e-6 if precision else 2e-3), (err, res, iters)


def test_chebyshev_pcg_reaches_newton_tolerance_full_size(ttie):
    """The crossing cloth's Newton system: the Chebyshev-preconditioned PCG (what AUTO picks
    there) reaches the Newton step's relative tolerance (1e-3) within the iteration cap, in fewer
    iterations than block Jacobi."""
    m = ti.cloth(256, seed=2).as_f32()
    x0, tri, _ = _dev(m)
    it = {}
    for pc in (ttie.PCG_BLOCK_JACOBI, ttie.PCG_CHEBYSHEV, ttie.PCG_AUTO):
        x = x0.clone()
        ctx = ttie.Context(pcg_precond=pc)
        ctx.build_bvh(x, tri)
        info = ctx.newton_step(x)
        it[pc] = (info["pcg_iters"], info["pcg_rel_residual"])
        assert np.isfinite(info["energy_new"]) and info["grad_dot_dir"] < 0
    assert it[ttie.PCG_CHEBYSHEV][1] <= 1e-3 and it[ttie.PCG_CHEBYSHEV][0] < 200, it
    assert it[ttie.PCG_CHEBYSHEV][0] < it[ttie.PCG_BLOCK_JACOBI][0], it
    assert it[ttie.PCG_AUTO] == it[ttie.PCG_CHEBYSHEV], it
