"""ttie_pcg_static: the PCG solve without any device allocation, for callers that
cannot allocate (a fixed, pre-planned device-memory budget; no cudaMalloc allowed).

Called through the C ABI with a system assembled by the library and compared with
the allocating ttie_pcg on the same system, on two calls in a row (the static work
array keeps the previous call's contents, so the second call checks that it clears
what must start at zero).  This file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _declare(L):
    f = L.ttie_pcg_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    return L


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06511_gb300 import ttie
    return _declare(ttie.load())


def _system():
    import ttie_inputs as ti
    from paper_2606_06511_gb300 import ttie
    m = ti.cloth(40, seed=2, shear=0.3).as_f32()
    x = torch.tensor(m.x, dtype=torch.float32, device="cuda")
    tri = torch.tensor(m.tri, dtype=torch.int32, device="cuda")
    ctx = ttie.Context()
    ctx.build_bvh(x, tri)
    ctx.eval_pairs(x, ttie.EVAL_E | ttie.EVAL_H)
    bsr = ctx.assemble()
    return ctx, bsr


def _call(lib, bsr, mu, rhs, rtol, max_it, n_rows=None):
    out = torch.full_like(rhs, float("nan"))
    it = ctypes.c_int()
    rel = ctypes.c_double()
    n = bsr.vertex_of_row.numel() if n_rows is None else n_rows
    s = lib.ttie_pcg_static(bsr.row_ptr.data_ptr(), bsr.col_idx.data_ptr(), bsr.val.data_ptr(), n, mu,
                            rhs.data_ptr(), out.data_ptr(), rtol, max_it,
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(it),
                            ctypes.byref(rel))
    return s, out, it.value, rel.value


def _bsr_matvec(rp, ci, val, mu, x):
    """(H + mu I) x in FP64 from the block-CSR arrays."""
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    y = mu * x.copy()
    np.add.at(y, rows, np.einsum("bij,bj->bi", val, x[ci]))
    return y


def test_static_pcg_matches_allocating_pcg(lib):
    from paper_2606_06511_gb300 import ttie
    ctx, bsr = _system()
    n = bsr.vertex_of_row.numel()
    assert 0 < n <= 16384
    rhs = (-bsr.grad).contiguous()
    rtol, max_it = 1e-4, 2000
    ref, it_ref, rel_ref = ctx.pcg(rhs, rtol=rtol, max_it=max_it)
    assert rel_ref <= rtol
    # the context's regulariser, mu_rel * trace(H+) / (3 n_rows), from the diagonal blocks
    rp = bsr.row_ptr.cpu().numpy()
    ci = bsr.col_idx.cpu().numpy()
    val = bsr.val.double().cpu().numpy()
    rows = np.repeat(np.arange(n), np.diff(rp))
    mu = ctx.params.mu_rel * np.trace(val[rows == ci], axis1=1, axis2=2).sum() / (3.0 * n)
    b = rhs.double().cpu().numpy().reshape(-1, 3)
    nb = np.linalg.norm(b)
    refn = ref.double().cpu().numpy()
    # same tolerance as the allocating solver's test: residual at the requested level up
    # to FP32 rounding of the product, and the two answers agree in the residual norm
    assert np.linalg.norm(_bsr_matvec(rp, ci, val, mu, refn) - b) <= 1e-2 * nb
    for call in range(2):   # two calls in a row share the static work array
        s, out, it, rel = _call(lib, bsr, mu, rhs, rtol, max_it)
        assert s == ttie.TTIE_OK
        assert rel <= rtol and it > 0
        o = out.double().cpu().numpy()
        assert np.isfinite(o).all()
        assert np.linalg.norm(_bsr_matvec(rp, ci, val, mu, o) - b) <= 1e-2 * nb, call
        assert np.linalg.norm(_bsr_matvec(rp, ci, val, mu, o - refn)) <= 2e-2 * nb, call


def test_static_pcg_rejects_oversize(lib):
    from paper_2606_06511_gb300 import ttie
    _, bsr = _system()
    rhs = (-bsr.grad).contiguous()
    s, out, _, _ = _call(lib, bsr, 1e-6, rhs, 1e-5, 10, n_rows=16385)
    assert s == ttie.TTIE_ERR_INVALID
    assert torch.isnan(out).all()   # nothing was written


def test_static_pcg_in_the_self_checking_build(lib):
    """The self-checking build (bounds checks against the block count read from row_ptr[n_rows],
    a synchronisation after each launch) of the entry point accepts a valid system: TTIE_OK,
    finite output, the same answer as the allocating solver within the tolerance above.  The
    checked library is a separate file loaded beside the normal one; the system comes from the
    normal library."""
    from paper_2606_06511_gb300 import ttie
    from paper_2606_06511_gb300.build import build as build_lib
    checked = _declare(ctypes.CDLL(build_lib(checked=True)))
    ctx, bsr = _system()
    n = bsr.vertex_of_row.numel()
    rhs = (-bsr.grad).contiguous()
    ref, _, _ = ctx.pcg(rhs, rtol=1e-4, max_it=2000)
    rp = bsr.row_ptr.cpu().numpy()
    ci = bsr.col_idx.cpu().numpy()
    val = bsr.val.double().cpu().numpy()
    rows = np.repeat(np.arange(n), np.diff(rp))
    mu = ctx.params.mu_rel * np.trace(val[rows == ci], axis1=1, axis2=2).sum() / (3.0 * n)
    b = rhs.double().cpu().numpy().reshape(-1, 3)
    nb = np.linalg.norm(b)
    for call in range(2):
        s, out, it, rel = _call(checked, bsr, mu, rhs, 1e-4, 2000)
        assert s == ttie.TTIE_OK, call
        o = out.double().cpu().numpy()
        assert np.isfinite(o).all() and rel <= 1e-4 and it > 0
        assert np.linalg.norm(_bsr_matvec(rp, ci, val, mu, o) - b) <= 1e-2 * nb, call
        assert np.linalg.norm(_bsr_matvec(rp, ci, val, mu, o - ref.double().cpu().numpy())) <= 2e-2 * nb, call
