"""Elastic term of the quasi-static simulation (mass-spring springs and anchors, Fig. 2) on the
GPU against the FP64 oracle: the energies of a Newton step, the direction of the combined
system (H+ of pairs, springs and anchors + mu I) d = -g, a simulation from an intersecting
state to a certified valid one, and the argument errors."""
import numpy as np
import pytest
import torch

import oracle as O
import ttie_inputs as ti

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ttie():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06511_gb300 import ttie as t
    return t


def _prestressed(m, seed=3):
    """Springs on every edge with rest lengths 0.8 .. 1.2 times their length (stretched and
    compressed: the projection clamps the compressed ones), three anchors pulled aside."""
    rng = np.random.default_rng(seed)
    e = ti.edge_list(m.tri)
    rest = rng.uniform(0.8, 1.2, len(e)) * np.linalg.norm(m.x[e[:, 0]] - m.x[e[:, 1]], axis=1)
    anchors = rng.choice(m.V, 3, replace=False).astype(np.int32)
    targets = m.x[anchors] + 0.02 * rng.standard_normal((3, 3))
    return O.Elastic(e, rest, 0.5, anchors, targets, 2.0)


def _set(ctx, el, dt):
    dev = lambda a, t: torch.tensor(a, dtype=t, device="cuda")
    ctx.set_elastic(dev(el.edges, torch.int32), dev(el.rest, dt), el.k_edge, dev(el.anchors, torch.int32),
                    dev(el.targets, dt), el.k_anchor)


def test_elastic_step_matches_oracle(ttie):
    m = ti.cloth(12, seed=21)
    el = _prestressed(m)
    prm = O.NewtonParams(max_step=0.0)
    E, n, grad, d, rows = O.newton_direction_elastic(m.x, m.tri, None, prm, el)
    assert n > 0
    x = torch.tensor(m.x, dtype=torch.float64, device="cuda")
    tri = torch.tensor(m.tri, dtype=torch.int32, device="cuda")
    ctx = ttie.Context(precision=ttie.F64, pcg_rtol=1e-11, pcg_max_it=5000, max_step=0.0)
    ctx.build_bvh(x, tri)
    _set(ctx, el, torch.float64)
    info = ctx.newton_step(x.clone())
    assert info["n_active"] == n
    assert info["energy"] == pytest.approx(E, rel=1e-10)
    assert info["energy_elastic"] == pytest.approx(O.elastic_energy(m.x, el), rel=1e-10)
    assert info["n_rows"] == len(rows)
    got = ctx.get_direction().cpu().numpy()
    assert np.abs(got - d).max() <= 1e-7 * np.abs(d).max()
    assert info["grad_dot_dir"] == pytest.approx(float(np.sum(grad * d)), rel=1e-7)


def test_elastic_step_f32_matches_oracle(ttie):
    m = ti.cloth(12, seed=21)
    el = _prestressed(m)
    prm = O.NewtonParams(max_step=0.0)
    E, n, grad, d, rows = O.newton_direction_elastic(m.x, m.tri, None, prm, el)
    x = torch.tensor(m.x, dtype=torch.float32, device="cuda")
    tri = torch.tensor(m.tri, dtype=torch.int32, device="cuda")
    ctx = ttie.Context(pcg_rtol=1e-6, pcg_max_it=5000, max_step=0.0)
    ctx.build_bvh(x, tri)
    _set(ctx, el, torch.float32)
    info = ctx.newton_step(x.clone())
    assert info["n_active"] == n and info["n_rows"] == len(rows)
    assert info["energy"] == pytest.approx(E, rel=1e-4)
    # FP32 positions, FP32 solve to 1e-6: the direction within cond-limited FP32 accuracy
    got = ctx.get_direction().double().cpu().numpy()
    assert np.linalg.norm(got - d) <= 2e-2 * np.linalg.norm(d)


def test_removing_the_term_restores_the_plain_step(ttie):
    m = ti.cloth(12, seed=21)
    x0 = torch.tensor(m.x, dtype=torch.float32, device="cuda")
    tri = torch.tensor(m.tri, dtype=torch.int32, device="cuda")
    outs = []
    for with_term in (False, True):
        ctx = ttie.Context()
        x = x0.clone()
        ctx.build_bvh(x, tri)
        if with_term:
            _set(ctx, _prestressed(m), torch.float32)
            ctx.set_elastic()
        outs.append((ctx.newton_step(x), x.cpu()))
    assert torch.equal(outs[0][1], outs[1][1])
    assert outs[1][0]["energy_elastic"] == 0.0


def test_quasi_static_simulation_reaches_valid_state(ttie):
    """Fig. 2: from an intersecting state to a valid one.  Two unit icospheres overlapping by
    0.05, springs on every edge at rest (k = 0.1, about a tenth of the mean diagonal of the
    pairs' H+ at the start): the solve separates them with little distortion, and the exact
    oracle certifies the end state."""
    m = ti.two_icospheres(offset=(1.95, 0.0, 0.0)).as_f32()
    e = ti.edge_list(m.tri)
    rest = np.linalg.norm(m.x[e[:, 0]] - m.x[e[:, 1]], axis=1)
    x = torch.tensor(m.x, dtype=torch.float32, device="cuda")
    tri = torch.tensor(m.tri, dtype=torch.int32, device="cuda")
    grp = torch.tensor(m.group, dtype=torch.int32, device="cuda")
    ctx = ttie.Context(pair_mode=1, newton_max_it=40)
    ctx.build_bvh(x, tri, grp)
    ctx.set_elastic(torch.tensor(e, device="cuda"), torch.tensor(rest, dtype=torch.float32, device="cuda"), 0.1)
    info = ctx.solve(x)
    assert info["converged"] == 1, info
    xf = x.double().cpu().numpy()
    assert O.certify(xf, m.tri, m.group, "inter") == 0
    strain = np.abs(np.linalg.norm(xf[e[:, 0]] - xf[e[:, 1]], axis=1) / rest - 1).max()
    assert strain < 0.05
    # the oracle's simulation (FP64) of the same state takes about as many iterations
    _, it_o, ok_o = O.quasi_static_solve(m.x.astype(np.float64), m.tri, m.group,
                                         O.NewtonParams(newton_max_it=40, mode="inter"),
                                         O.Elastic(e, rest.astype(np.float64), 0.1))
    assert ok_o and abs(info["iterations"] - it_o) <= 3


def test_elastic_errors(ttie):
    m = ti.cloth(8, seed=1)
    x = torch.tensor(m.x, dtype=torch.float32, device="cuda")
    tri = torch.tensor(m.tri, dtype=torch.int32, device="cuda")
    e = torch.tensor(ti.edge_list(m.tri), device="cuda")
    rest = torch.ones(e.shape[0], dtype=torch.float32, device="cuda")
    ctx = ttie.Context()
    with pytest.raises(ttie.TTIEError) as err:
        ctx.set_elastic(e, rest, 1.0)
    assert err.value.status == ttie.TTIE_ERR_STATE
    ctx.build_bvh(x, tri)
    bad = e.clone()
    bad[3, 1] = m.V
    with pytest.raises(ttie.TTIEError) as err:
        ctx.set_elastic(bad, rest, 1.0)
    assert err.value.status == ttie.TTIE_ERR_INVALID
    bad = e.clone()
    bad[3, 1] = bad[3, 0]
    with pytest.raises(ttie.TTIEError) as err:
        ctx.set_elastic(bad, rest, 1.0)
    assert err.value.status == ttie.TTIE_ERR_INVALID
    with pytest.raises(ttie.TTIEError) as err:
        ctx.set_elastic(e, rest, -1.0)
    assert err.value.status == ttie.TTIE_ERR_INVALID
    with pytest.raises(ttie.TTIEError) as err:
        ctx.set_elastic(e, rest.double(), 1.0)
    assert err.value.status == ttie.TTIE_ERR_INVALID
    ctx.set_elastic(e, rest, 1.0)          # valid after the errors
    ctx.newton_step(x)
    # batched instances do not take the term
    mb, vo, to = ti.ellipsoid_batch(2, seed=4, f_min=60, f_max=200)
    xb = torch.tensor(mb.x, dtype=torch.float32, device="cuda")
    tb = torch.tensor(mb.tri, dtype=torch.int32, device="cuda")
    gb = torch.tensor(mb.group, dtype=torch.int32, device="cuda")
    cb = ttie.Context(pair_mode=2)
    cb.build_bvh(xb, tb, gb)
    eb = torch.tensor(ti.edge_list(mb.tri), device="cuda")
    with pytest.raises(ttie.TTIEError) as err:
        cb.set_elastic(eb, torch.ones(eb.shape[0], dtype=torch.float32, device="cuda"), 1.0)
    assert err.value.status == ttie.TTIE_ERR_INVALID
