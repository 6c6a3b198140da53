"""Second order through the C ABI: the exact Hessian-vector product (forward-mode duals
through the Eq. 3 pair gradient) and the PSD product H+ v on the assembled system, against
the oracle; and the torch.autograd wrapper (energy, gradient, double backward).

Tolerances.  FP64: the oracle's product is a fourth-order central difference of its FP64
gradient (relative accuracy about 1e-7), so 1e-5 of the largest entry.  FP32: second
derivatives of t_c divide by the same near-parallel normal products as the gradient, so the
FP32 position rounding (2^-24 of the pair's size) is amplified once more; the check is
norm-wise, 2e-3 of the oracle's norm, plus the identities below, which are exact.
Identities of any correct Hessian of a degree-4, rigid-motion-invariant energy:
H (x - c) = 3 g,  H (w x x) = w x g,  H 1 = 0.
"""
import numpy as np
import pytest
import torch

import oracle as O
import ttie_inputs as ti
from _cases import MODE, small_cases

pytestmark = pytest.mark.gpu

CASES = small_cases()
NAMES = ["cloth40", "soup", "tori", "spheres_inter"]


@pytest.fixture(scope="module")
def ttie():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06511_gb300 import ttie as t
    return t


def _setup(ttie, name, precision):
    m, mode = CASES[name]
    dt = torch.float64 if precision == ttie.F64 else torch.float32
    x = torch.tensor(m.x, dtype=dt, device="cuda")
    tri = torch.tensor(m.tri, dtype=torch.int32, device="cuda")
    grp = torch.tensor(m.group, dtype=torch.int32, device="cuda")
    ctx = ttie.Context(precision=precision, pair_mode=MODE[mode])
    ctx.build_bvh(x, tri, grp)
    g = torch.empty_like(x)
    E, n_act = ctx.eval_pairs(x, ttie.EVAL_E | ttie.EVAL_G | ttie.EVAL_H, grad=g)
    return m, mode, x, ctx, g, n_act


_oracle_cache = {}


def _oracle(name):
    if name not in _oracle_cache:
        m, mode = CASES[name]
        pairs = O.candidate_pairs(m.x, m.tri, m.group, mode)
        _oracle_cache[name] = O.evaluate(m.x, m.tri, pairs)
    return _oracle_cache[name]


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_exact_hvp_matches_oracle(ttie, name, prec):
    precision = ttie.F64 if prec == "f64" else ttie.F32
    m, mode, x, ctx, g, n_act = _setup(ttie, name, precision)
    ev = _oracle(name)
    assert n_act == int(ev.active.sum()) and n_act > 0
    rng = np.random.default_rng(3)
    v = rng.normal(size=m.x.shape)
    hv = ctx.hvp(x, torch.tensor(v, dtype=x.dtype, device="cuda"), exact=True).double().cpu().numpy()
    ho = O.hessian_vector_product(m.x, m.tri, ev, v)
    scale = np.abs(ho).max()
    assert scale > 0
    if prec == "f64":
        assert np.abs(hv - ho).max() <= 1e-5 * scale
    else:
        assert np.linalg.norm(hv - ho) <= 2e-3 * np.linalg.norm(ho)
    # vertices outside every intersecting pair get exactly zero
    used = np.zeros(m.V, bool)
    act = ev.pairs[ev.active]
    used[O.pair_dofs(m.tri, act).ravel()] = True
    assert np.all(hv[~used] == 0)


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_exact_hvp_identities(ttie, name, prec):
    precision = ttie.F64 if prec == "f64" else ttie.F32
    m, mode, x, ctx, g, n_act = _setup(ttie, name, precision)
    tol = 1e-8 if prec == "f64" else 2e-3
    gn = g.double().cpu().numpy()
    gs = np.abs(gn).max()
    xd = x.double()
    c = xd.mean(0, keepdim=True)
    h_scale = ctx.hvp(x, (xd - c).to(x.dtype), exact=True).double().cpu().numpy()
    assert np.abs(h_scale - 3 * gn).max() <= tol * 3 * gs
    w = torch.tensor([0.3, -0.7, 0.5], dtype=torch.float64, device="cuda")
    h_rot = ctx.hvp(x, torch.cross(w.expand_as(xd), xd - c, dim=1).to(x.dtype), exact=True).double().cpu().numpy()
    assert np.abs(h_rot - np.cross(w.cpu().numpy(), gn)).max() <= tol * 10 * gs
    one = torch.ones_like(x)
    h_tr = ctx.hvp(x, one, exact=True).double().cpu().numpy()
    lin = np.abs(ctx.hvp(x, (xd - c).to(x.dtype) / (xd - c).abs().max(), exact=True).double().cpu().numpy()).max()
    assert np.abs(h_tr).max() <= tol * 10 * lin


@pytest.mark.parametrize("name", NAMES)
def test_psd_hvp_matches_assembled_blocks(ttie, name):
    m, mode, x, ctx, g, n_act = _setup(ttie, name, ttie.F64)
    ev = _oracle(name)
    rng = np.random.default_rng(4)
    v = rng.normal(size=m.x.shape)
    hv = ctx.hvp(x, torch.tensor(v, device="cuda"), exact=False).cpu().numpy()
    _, blocks = O.assemble(m.tri, ev, m.V)
    ho = np.zeros_like(v)
    for (r, c), b in blocks.items():
        ho[r] += b @ v[c]
    scale = np.abs(ho).max()
    assert np.abs(hv - ho).max() <= 1e-4 * scale
    assert float((v * hv).sum()) >= -1e-10 * scale * np.abs(v).sum()   # H+ is PSD


def test_hvp_before_eval_is_a_state_error(ttie):
    m, _ = CASES["soup"]
    x = torch.tensor(m.x, dtype=torch.float32, device="cuda")
    ctx = ttie.Context()
    with pytest.raises(ttie.TTIEError) as e:
        ctx.hvp(x, torch.zeros_like(x))
    assert e.value.status == ttie.TTIE_ERR_STATE


def test_hvp_no_active_pairs(ttie):
    m = ti.icosphere(2).as_f32()
    x = torch.tensor(m.x, dtype=torch.float32, device="cuda")
    tri = torch.tensor(m.tri, dtype=torch.int32, device="cuda")
    ctx = ttie.Context()
    ctx.build_bvh(x, tri)
    E, n = ctx.eval_pairs(x, ttie.EVAL_E | ttie.EVAL_H)
    assert n == 0
    for exact in (True, False):
        out = ctx.hvp(x, torch.ones_like(x), exact=exact)
        assert torch.count_nonzero(out) == 0


# ----------------------------------------------------------------- autograd
def _energy_fn(ttie, m, mode, precision):
    from paper_2606_06511_gb300.autograd import TTIEnergy
    tri = torch.tensor(m.tri, dtype=torch.int32, device="cuda")
    grp = torch.tensor(m.group, dtype=torch.int32, device="cuda")
    return TTIEnergy(tri, grp, precision=precision, pair_mode=MODE[mode])


def test_autograd_energy_gradient_and_double_backward(ttie):
    m, mode = CASES["tori"]
    f = _energy_fn(ttie, m, mode, ttie.F64)
    x = torch.tensor(m.x, dtype=torch.float64, device="cuda", requires_grad=True)
    E = f(x)
    (g,) = torch.autograd.grad(E, x, create_graph=True)
    ev = _oracle("tori")
    assert E.item() == pytest.approx(float(ev.T.sum()), rel=1e-9)
    go, _ = O.assemble(m.tri, ev, m.V)
    assert np.abs(g.detach().cpu().numpy() - go).max() <= 1e-6 * np.abs(go).max()
    rng = np.random.default_rng(5)
    v = torch.tensor(rng.normal(size=m.x.shape), device="cuda")
    (hv,) = torch.autograd.grad((g * v).sum(), x)
    ho = O.hessian_vector_product(m.x, m.tri, ev, v.cpu().numpy())
    assert np.abs(hv.cpu().numpy() - ho).max() <= 1e-5 * np.abs(ho).max()
    # scaling the output scales both orders
    (g2,) = torch.autograd.grad(2.5 * f(x), x)
    assert torch.allclose(g2, 2.5 * g.detach(), rtol=1e-12, atol=0)


def test_autograd_gradcheck_fp64(ttie):
    m = ti.triangle_soup(40, seed=21, size=0.6)
    f = _energy_fn(ttie, m, "self", ttie.F64)
    x = torch.tensor(m.x, dtype=torch.float64, device="cuda", requires_grad=True)
    assert f.__call__(x).item() > 0 and f.last > 5
    assert torch.autograd.gradcheck(f, (x,), eps=1e-6, atol=1e-6, rtol=1e-5, fast_mode=True)
    assert torch.autograd.gradgradcheck(f, (x,), eps=1e-6, atol=1e-5, rtol=1e-4, fast_mode=True)


def _first_active_pairs_submesh(ttie, m, n_pairs):
    """The triangles of the first n_pairs intersecting pairs by key (i, j) of mesh m, as a mesh of
    their own (vertices renumbered), with the keys."""
    x = torch.tensor(m.x, dtype=torch.float64, device="cuda")
    tri = torch.tensor(m.tri, dtype=torch.int32, device="cuda")
    ctx = ttie.Context(precision=ttie.F64)
    ctx.build_bvh(x, tri)
    ctx.eval_pairs(x, ttie.EVAL_E)
    ap, _, _ = ctx.get_active(with_derivatives=False)
    ap = ap.cpu().numpy().astype(np.int64)
    ap = ap[np.lexsort((ap[:, 1], ap[:, 0]))][:n_pairs]
    keep = np.unique(ap.ravel())
    sub_tri = m.tri[keep]
    used = np.unique(sub_tri)
    remap = -np.ones(m.V, np.int64)
    remap[used] = np.arange(len(used))
    return ti.Mesh(m.x[used], remap[sub_tri].astype(np.int32), np.zeros(len(keep), np.int32)), ap


def test_gradcheck_on_interlocked_tori_full_size(ttie):
    """The tori workload at full size (2 x 65,536 triangles, tubes interpenetrating at offset 0.5,
    jitter 0.005): the triangles of its first 1,000 intersecting pairs by key, in FP64, pass
    gradcheck and gradgradcheck of the autograd energy (exact Hessian-vector products in the
    double backward), and the exact Hessian-vector product matches central differences of the
    library's gradient along a random direction."""
    m = ti.interlocked_tori(offset=(0.5, 0, 0))
    assert m.F == 2 * 65536
    sub, keys = _first_active_pairs_submesh(ttie, m, 1000)
    assert len(keys) == 1000
    f = _energy_fn(ttie, sub, "self", ttie.F64)
    x = torch.tensor(sub.x, dtype=torch.float64, device="cuda", requires_grad=True)
    assert f(x).item() > 0 and f.last >= 1000
    assert torch.autograd.gradcheck(f, (x,), eps=1e-7, atol=1e-7, rtol=1e-5, fast_mode=True)
    assert torch.autograd.gradgradcheck(f, (x,), eps=1e-7, atol=1e-6, rtol=1e-4, fast_mode=True)
    # exact HVP against central differences of the gradient (4th order), step 1e-6 of an edge
    ctx = ttie.Context(precision=ttie.F64)
    xd = x.detach()
    tri = torch.tensor(sub.tri, dtype=torch.int32, device="cuda")
    rng = np.random.default_rng(9)
    v = torch.tensor(rng.normal(size=sub.x.shape), device="cuda")

    def grad_at(xx):
        ctx.build_bvh(xx, tri)
        g = torch.zeros_like(xx)
        ctx.eval_pairs(xx, ttie.EVAL_E | ttie.EVAL_G, grad=g)
        return g
    ctx.build_bvh(xd, tri)
    ctx.eval_pairs(xd, ttie.EVAL_E | ttie.EVAL_H)
    hv = ctx.hvp(xd, v, exact=True)
    h = 2e-8
    fd = (8 * (grad_at(xd + h * v) - grad_at(xd - h * v)) - (grad_at(xd + 2 * h * v) - grad_at(xd - 2 * h * v))) / (12 * h)
    err = (hv - fd).abs().max().item() / hv.abs().max().item()
    assert err <= 1e-4, err


def test_adam_descends_on_linked_tori(ttie):
    """The energy as a loss for a first-order optimizer: Adam (lr 1e-3) on sum T over
    interpenetrating linked tori (2 x 8192 triangles) lowers the energy at least fourfold
    within 100 steps.  (First-order descent does not reach an intersection-free state; the
    Newton route does that.)"""
    m = ti.interlocked_tori(offset=(0.5, 0, 0), n_major=128, n_minor=64).as_f32()
    f = _energy_fn(ttie, m, "self", ttie.F32)
    x = torch.tensor(m.x, dtype=torch.float32, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([x], lr=1e-3)
    hist = []
    for it in range(101):
        opt.zero_grad()
        E = f(x)
        E.backward()
        opt.step()
        hist.append((E.item(), f.last))
        assert np.isfinite(hist[-1][0])
    assert hist[0][1] > 100
    assert hist[-1][0] < 0.25 * hist[0][0]


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_dual_gradients_match_analytic_chain_rule(ttie, name, prec):
    """Forward-mode duals in FP64 on the GPU (the appendix's route) against the analytic
    gradients of t_c from the evaluation (FP64: 1e-7 of each pair's largest entry; FP32
    positions: the stated 1e-4 for gradients, every pair) and against the oracle."""
    precision = ttie.F64 if prec == "f64" else ttie.F32
    m, mode, x, ctx, g, n_act = _setup(ttie, name, precision)
    dual = ctx.dual_gradients(x).cpu().numpy()
    pairs, tc, dtc = ctx.get_active()
    dtc = dtc.double().cpu().numpy()
    assert dual.shape == dtc.shape and len(dual) == n_act
    ev = _oracle(name)
    act = ev.pairs[ev.active]
    idx = {tuple(p): k for k, p in enumerate(act.tolist())}
    k = np.array([idx[tuple(p)] for p in pairs.cpu().numpy().astype(np.int64).tolist()])
    od = ev.dtc[ev.active][k]
    scale = np.abs(od).max(axis=2, keepdims=True)
    # the dual evaluation reads the stored positions, so it matches the oracle to FP64 rounding
    assert (np.abs(dual - od) <= 1e-7 * scale).all()
    tol = 1e-7 if prec == "f64" else 1e-4
    err = (np.abs(dtc - dual) / scale).max()
    assert err <= tol, err
