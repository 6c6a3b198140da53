"""Python binding of libttie (ctypes; argument marshalling only).

Every computation runs in the CUDA kernels of ``libttie.so``; this module only
checks tensors, passes device pointers and the current torch stream, and turns
status codes into exceptions.  It raises ``TTIEError`` when the library is
missing: there is no CPU fallback.

Names follow the C ABI in ``include/ttie.h``: ``Context.build_bvh``,
``eval_pairs``, ``assemble``, ``pcg``, ``newton_step``, ``solve`` and the
inspection calls.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libttie.so")

TTIE_OK, TTIE_ERR_INVALID, TTIE_ERR_CUDA, TTIE_ERR_OOM, TTIE_ERR_CAPACITY, TTIE_ERR_NONFINITE, \
    TTIE_ERR_NOT_CONVERGED, TTIE_ERR_STATE = range(8)
STATUS_NAMES = ["OK", "INVALID", "CUDA", "OOM", "CAPACITY", "NONFINITE", "NOT_CONVERGED", "STATE"]
F32, F64 = 0, 1
PAIRS_SELF, PAIRS_INTER_GROUP, PAIRS_INTRA_GROUP, PAIRS_BRUTE, PAIRS_HASH = 0, 1, 2, 4, 8
PSD_PER_PART, PSD_DROP_CROSS, PSD_WHOLE = 0, 1, 2
PCG_BLOCK_JACOBI, PCG_CHEBYSHEV, PCG_AUTO = 0, 1, 2
TRAVERSAL_TWO_WALKS, TRAVERSAL_ONE_WALK = 0, 1
LS_ARMIJO, LS_FEWER = 0, 1
PCG_KERNEL_AUTO, PCG_KERNEL_RESIDENT, PCG_KERNEL_STREAMED, PCG_KERNEL_RESIDENT_UNCACHED = 0, 1, 2, 3
EVAL_E, EVAL_G, EVAL_H = 1, 2, 4


class TTIEError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("TTIE_%s: %s" % (name, msg))


class Params(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("pair_mode", ctypes.c_int), ("psd_mode", ctypes.c_int),
                ("tc_scale", ctypes.c_double), ("mu_rel", ctypes.c_double), ("pcg_rtol", ctypes.c_double),
                ("pcg_max_it", ctypes.c_int), ("newton_max_it", ctypes.c_int), ("ls_max_halvings", ctypes.c_int),
                ("armijo_c", ctypes.c_double), ("push_eta", ctypes.c_double), ("exact_only", ctypes.c_int),
                ("profile", ctypes.c_int), ("max_step", ctypes.c_double), ("max_candidates", ctypes.c_int64),
                ("inst_threads", ctypes.c_int), ("test_withhold", ctypes.c_int), ("pcg_precond", ctypes.c_int),
                ("pcg_cheb_degree", ctypes.c_int), ("traversal_mode", ctypes.c_int),
                ("ls_rule", ctypes.c_int), ("push_eta_max", ctypes.c_double), ("pcg_kernel", ctypes.c_int)]


class BsrView(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("nnzb", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p), ("vertex_of_row", ctypes.c_void_p),
                ("grad", ctypes.c_void_p)]


class StepInfo(ctypes.Structure):
    _fields_ = [("n_candidates", ctypes.c_int64), ("n_active", ctypes.c_int64), ("n_rows", ctypes.c_int64),
                ("nnzb", ctypes.c_int64), ("energy", ctypes.c_double), ("energy_new", ctypes.c_double),
                ("n_active_new", ctypes.c_int64), ("alpha", ctypes.c_double), ("grad_dot_dir", ctypes.c_double),
                ("pcg_iters", ctypes.c_int), ("pcg_rel_residual", ctypes.c_double), ("ls_trials", ctypes.c_int),
                ("n_candidates_swept", ctypes.c_int64), ("ms_build", ctypes.c_float), ("ms_eval", ctypes.c_float),
                ("ms_assemble", ctypes.c_float), ("ms_pcg", ctypes.c_float), ("ms_line_search", ctypes.c_float),
                ("ms_classify", ctypes.c_float), ("ms_pcg_kernel", ctypes.c_float),
                ("pcg_block_iters", ctypes.c_int64), ("pcg_row_iters", ctypes.c_int64),
                ("energy_elastic", ctypes.c_double), ("pcg_kernel", ctypes.c_int),
                ("stage_launches", ctypes.c_int64 * 5), ("inst_threads", ctypes.c_int),
                ("inst_blocks_per_sm", ctypes.c_int), ("inst_order", ctypes.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["stage_launches"] = list(self.stage_launches)
        return d


class Elastic(ctypes.Structure):
    """ttie_elastic: springs k_edge/2 (|x_i - x_j| - rest)^2 and anchors k_anchor/2 |x_a - t_a|^2."""
    _fields_ = [("edges", ctypes.c_void_p), ("rest", ctypes.c_void_p), ("n_edges", ctypes.c_int64),
                ("k_edge", ctypes.c_double), ("anchors", ctypes.c_void_p), ("targets", ctypes.c_void_p),
                ("n_anchors", ctypes.c_int64), ("k_anchor", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("n_active_initial", ctypes.c_int64),
                ("n_active_final", ctypes.c_int64), ("energy_initial", ctypes.c_double),
                ("energy_final", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

_SIGS = {
    "ttie_default_params": (None, [ctypes.POINTER(Params)]),
    "ttie_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Params), ctypes.c_void_p]),
    "ttie_destroy": (None, [ctypes.c_void_p]),
    "ttie_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "ttie_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Params)]),
    "ttie_build_bvh": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "ttie_eval_pairs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]),
    "ttie_assemble": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(BsrView)]),
    "ttie_copy_bsr": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 5),
    "ttie_pcg": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "ttie_newton_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(StepInfo)]),
    "ttie_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(SolveInfo)]),
    "ttie_get_candidates": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_int64)]),
    "ttie_get_active": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "ttie_get_direction": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "ttie_get_filter_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "ttie_struct_sizes": (None, [ctypes.POINTER(ctypes.c_int64)]),
    "ttie_get_launch_count": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "ttie_hvp": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "ttie_dual_gradients": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ttie_set_elastic": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Elastic)]),
}


def load(path: str = LIB_PATH):
    """Load libttie.so (built by ``paper_2606_06511_gb300.build``); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise TTIEError(TTIE_ERR_STATE, "libttie.so not built (%s); run __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def default_params(**kw) -> Params:
    p = Params()
    load().ttie_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError("unknown parameter %s" % k)
        setattr(p, k, v)
    return p


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _check_dev(t, name, dtype=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TTIEError(TTIE_ERR_INVALID, "%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise TTIEError(TTIE_ERR_INVALID, "%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise TTIEError(TTIE_ERR_INVALID, "%s must be %s, got %s" % (name, dtype, t.dtype))


@dataclass
class Bsr:
    row_ptr: torch.Tensor
    col_idx: torch.Tensor
    val: torch.Tensor          # [nnzb, 3, 3]
    vertex_of_row: torch.Tensor
    grad: torch.Tensor         # [n_rows, 3]


class Context:
    """One libttie context on the current CUDA device and torch stream."""

    def __init__(self, params: Params | None = None, stream=None, **kw):
        self.lib = load()
        self.params = params if params is not None else default_params(**kw)
        self.dtype = torch.float64 if self.params.precision == F64 else torch.float32
        st = stream if stream is not None else torch.cuda.current_stream()
        self.stream = st
        h = ctypes.c_void_p()
        s = self.lib.ttie_create(ctypes.byref(h), ctypes.byref(self.params), ctypes.c_void_p(st.cuda_stream))
        if s != TTIE_OK:
            raise TTIEError(s, "ttie_create failed")
        self.h = h
        self.V = None
        self.x_stride = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.ttie_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_x(self, x, name="x"):
        """Positions after ttie_build_bvh must have its layout: the library reads V x stride."""
        _check_dev(x, name, self.dtype)
        if self.V is not None and (x.dim() != 2 or tuple(x.shape) != (self.V, self.x_stride)):
            raise TTIEError(TTIE_ERR_INVALID, "%s must be [%d,%d] like the mesh given to build_bvh" %
                            (name, self.V, self.x_stride))

    def _chk(self, s):
        if s != TTIE_OK:
            raise TTIEError(s, self.lib.ttie_last_error(self.h).decode())
        return s

    def set_params(self, **kw):
        for k, v in kw.items():
            setattr(self.params, k, v)
        self._chk(self.lib.ttie_set_params(self.h, ctypes.byref(self.params)))

    # ---- C ABI calls
    def build_bvh(self, x: torch.Tensor, tri: torch.Tensor, group: torch.Tensor | None = None) -> int:
        _check_dev(x, "x", self.dtype)
        _check_dev(tri, "tri", torch.int32)
        if group is not None:
            _check_dev(group, "group", torch.int32)
        if x.dim() != 2 or x.shape[1] not in (3, 4) or tri.dim() != 2 or tri.shape[1] != 3:
            raise TTIEError(TTIE_ERR_INVALID, "x must be [V,3|4], tri [F,3]")
        n = ctypes.c_int64()
        self._chk(self.lib.ttie_build_bvh(self.h, _ptr(x), x.shape[0], x.shape[1], _ptr(tri), tri.shape[0],
                                          _ptr(group), ctypes.byref(n)))
        self.V = x.shape[0]
        self.x_stride = x.shape[1]
        return n.value

    def eval_pairs(self, x: torch.Tensor, what: int = EVAL_E, grad: torch.Tensor | None = None):
        """Returns (energy, n_active); fills ``grad`` ([V,3]) when given (needs EVAL_G)."""
        self._check_x(x)
        if grad is not None:
            _check_dev(grad, "grad", self.dtype)
            if tuple(grad.shape) != (x.shape[0], 3):
                raise TTIEError(TTIE_ERR_INVALID, "grad must be [V,3]")
        e = ctypes.c_double()
        n = ctypes.c_int64()
        self._chk(self.lib.ttie_eval_pairs(self.h, _ptr(x), what, ctypes.byref(e), ctypes.byref(n), _ptr(grad)))
        return e.value, n.value

    def assemble(self) -> Bsr:
        v = BsrView()
        self._chk(self.lib.ttie_assemble(self.h, ctypes.byref(v)))
        dev = torch.device("cuda", torch.cuda.current_device())
        rp = torch.empty(v.n_rows + 1, dtype=torch.int32, device=dev)
        ci = torch.empty(max(v.nnzb, 0), dtype=torch.int32, device=dev)
        val = torch.empty((max(v.nnzb, 0), 3, 3), dtype=self.dtype, device=dev)
        vr = torch.empty(v.n_rows, dtype=torch.int32, device=dev)
        g = torch.empty((v.n_rows, 3), dtype=self.dtype, device=dev)
        self._chk(self.lib.ttie_copy_bsr(self.h, _ptr(rp), _ptr(ci), _ptr(val), _ptr(vr), _ptr(g)))
        return Bsr(rp, ci, val, vr, g)

    def pcg(self, rhs: torch.Tensor, rtol: float = 1e-6, max_it: int = 1000):
        _check_dev(rhs, "rhs", self.dtype)
        out = torch.empty_like(rhs)
        it = ctypes.c_int()
        rr = ctypes.c_double()
        self._chk(self.lib.ttie_pcg(self.h, _ptr(rhs), _ptr(out), rtol, max_it, ctypes.byref(it), ctypes.byref(rr)))
        return out, it.value, rr.value

    def hvp(self, x: torch.Tensor, v: torch.Tensor, exact: bool = True) -> torch.Tensor:
        """Hessian of the energy (exact, or the assembled PSD H+) times v ([V,3]) at the positions
        of the last eval_pairs; x must be those positions."""
        self._check_x(x)
        _check_dev(v, "v", self.dtype)
        if tuple(v.shape) != (x.shape[0], 3):
            raise TTIEError(TTIE_ERR_INVALID, "v must be [V,3]")
        out = torch.empty_like(v)
        self._chk(self.lib.ttie_hvp(self.h, _ptr(x), _ptr(v), _ptr(out), 1 if exact else 0))
        return out

    def dual_gradients(self, x: torch.Tensor) -> torch.Tensor:
        """[n_active, 2, 18] float64 gradients of t_c^0, t_c^1 by forward-mode dual numbers (FP64) at
        the positions of the last eval_pairs (x must be those positions)."""
        self._check_x(x)
        n = ctypes.c_int64()
        self._chk(self.lib.ttie_get_active(self.h, None, None, None, 0, ctypes.byref(n)))
        out = torch.empty((max(n.value, 1), 2, 18), dtype=torch.float64, device="cuda")
        self._chk(self.lib.ttie_dual_gradients(self.h, _ptr(x), _ptr(out)))
        return out[: n.value]

    def set_elastic(self, edges: torch.Tensor | None = None, rest: torch.Tensor | None = None, k_edge: float = 0.0,
                    anchors: torch.Tensor | None = None, targets: torch.Tensor | None = None,
                    k_anchor: float = 0.0) -> None:
        """Elastic term of the quasi-static simulation (ttie_set_elastic): springs on edges
        [E,2] int32 with rest lengths [E] and anchors [A] int32 held at targets [A,3] (both in
        the context's dtype).  Called with no springs and no anchors it removes the term."""
        el = Elastic()
        keep = []
        if edges is not None and edges.numel():
            _check_dev(edges, "edges", torch.int32)
            _check_dev(rest, "rest", self.dtype)
            if edges.dim() != 2 or edges.shape[1] != 2 or tuple(rest.shape) != (edges.shape[0],):
                raise TTIEError(TTIE_ERR_INVALID, "edges must be [E,2] and rest [E]")
            el.edges, el.rest, el.n_edges, el.k_edge = _ptr(edges), _ptr(rest), edges.shape[0], float(k_edge)
            keep += [edges, rest]
        if anchors is not None and anchors.numel():
            _check_dev(anchors, "anchors", torch.int32)
            _check_dev(targets, "targets", self.dtype)
            if anchors.dim() != 1 or tuple(targets.shape) != (anchors.shape[0], 3):
                raise TTIEError(TTIE_ERR_INVALID, "anchors must be [A] and targets [A,3]")
            el.anchors, el.targets, el.n_anchors, el.k_anchor = _ptr(anchors), _ptr(targets), anchors.shape[0], \
                float(k_anchor)
            keep += [anchors, targets]
        self._chk(self.lib.ttie_set_elastic(self.h, ctypes.byref(el)))
        del keep   # the context copied the arrays during the call

    def newton_step(self, x: torch.Tensor) -> dict:
        self._check_x(x)
        info = StepInfo()
        self._chk(self.lib.ttie_newton_step(self.h, _ptr(x), ctypes.byref(info)))
        return info.as_dict()

    def solve(self, x: torch.Tensor, raise_on_limit: bool = False) -> dict:
        self._check_x(x)
        info = SolveInfo()
        s = self.lib.ttie_solve(self.h, _ptr(x), ctypes.byref(info))
        if s == TTIE_ERR_NOT_CONVERGED and not raise_on_limit:
            return info.as_dict()
        self._chk(s)
        return info.as_dict()

    # ---- inspection
    def get_candidates(self) -> torch.Tensor:
        n = ctypes.c_int64()
        self._chk(self.lib.ttie_get_candidates(self.h, None, 0, ctypes.byref(n)))
        out = torch.empty((n.value, 2), dtype=torch.int32, device="cuda")
        self._chk(self.lib.ttie_get_candidates(self.h, _ptr(out), n.value, ctypes.byref(n)))
        return out

    def get_active(self, with_derivatives: bool = True):
        n = ctypes.c_int64()
        self._chk(self.lib.ttie_get_active(self.h, None, None, None, 0, ctypes.byref(n)))
        pairs = torch.empty((n.value, 2), dtype=torch.int32, device="cuda")
        tc = dtc = None
        if with_derivatives:
            tc = torch.empty((n.value, 2), dtype=self.dtype, device="cuda")
            dtc = torch.empty((n.value, 2, 18), dtype=self.dtype, device="cuda")
        self._chk(self.lib.ttie_get_active(self.h, _ptr(pairs), _ptr(tc), _ptr(dtc), n.value, ctypes.byref(n)))
        return pairs, tc, dtc

    def get_direction(self) -> torch.Tensor:
        out = torch.empty((self.V, 3), dtype=self.dtype, device="cuda")
        self._chk(self.lib.ttie_get_direction(self.h, _ptr(out)))
        return out

    def get_filter_stats(self):
        arr = (ctypes.c_int64 * 3)()
        self._chk(self.lib.ttie_get_filter_stats(self.h, arr))
        return {"fp32": arr[0], "fp64": arr[1], "exact": arr[2]}

    def get_launch_count(self) -> int:
        n = ctypes.c_int64()
        self._chk(self.lib.ttie_get_launch_count(self.h, ctypes.byref(n)))
        return n.value
