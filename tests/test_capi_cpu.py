"""Host-side checks of the C ABI that need no GPU: the library builds, loads and
exports every entry point declared in include/ttie.h; arguments are rejected
before anything touches a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06511_gb300 import ttie
    return ttie.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ttie.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ttie_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_header_is_plain_c(tmp_path):
    """The boundary header compiles as strict C99 (and C++17) with every warning an error, so a
    C caller can use it; every declared entry point is referenced."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    names = declared_functions()
    src = tmp_path / "use_header.c"
    src.write_text('#include "ttie.h"\n' + "".join("void (*ref_%s)(void) = (void (*)(void))&%s;\n" % (n, n) for n in names) +
                   "int main(void) { ttie_params p; ttie_default_params(&p); return p.precision; }\n")
    for cmd in ([gcc, "-std=c99", "-pedantic"], [gcc, "-x", "c++", "-std=c++17"]):
        r = subprocess.run(cmd + ["-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), "-c", str(src),
                                  "-o", str(tmp_path / "use_header.o")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_default_params(lib):
    from paper_2606_06511_gb300 import ttie
    p = ttie.default_params()
    assert p.precision == ttie.F32 and p.pair_mode == ttie.PAIRS_SELF and p.psd_mode == ttie.PSD_PER_PART
    assert p.tc_scale == 1.0 and p.mu_rel == 1e-3 and p.push_eta == 0.5 and p.exact_only == 0
    # the fields appended last come back from the library's defaults: the binding's layout matches
    assert p.max_step == 1.0 and p.max_candidates == 0 and p.inst_threads == 0 and p.test_withhold == 0
    assert p.pcg_precond == ttie.PCG_AUTO and p.pcg_cheb_degree == 0
    assert p.traversal_mode == ttie.TRAVERSAL_ONE_WALK
    assert p.ls_rule == ttie.LS_ARMIJO and p.push_eta_max == 1.5 and p.pcg_kernel == ttie.PCG_KERNEL_AUTO


def test_null_context_is_rejected(lib):
    from paper_2606_06511_gb300 import ttie
    n = ctypes.c_int64()
    assert lib.ttie_build_bvh(None, None, 0, 3, None, 0, None, ctypes.byref(n)) == ttie.TTIE_ERR_INVALID
    assert lib.ttie_eval_pairs(None, None, 1, None, None, None) == ttie.TTIE_ERR_INVALID
    assert lib.ttie_newton_step(None, None, None) == ttie.TTIE_ERR_INVALID
    assert lib.ttie_last_error(None) == b"null context"
    assert lib.ttie_create(None, None, None) == ttie.TTIE_ERR_INVALID
    assert lib.ttie_set_elastic(None, None) == ttie.TTIE_ERR_INVALID


def test_bad_params_rejected_before_device(lib):
    from paper_2606_06511_gb300 import ttie
    h = ctypes.c_void_p()
    p = ttie.default_params(precision=7)
    assert lib.ttie_create(ctypes.byref(h), ctypes.byref(p), None) == ttie.TTIE_ERR_INVALID
    p = ttie.default_params(pair_mode=3)
    assert lib.ttie_create(ctypes.byref(h), ctypes.byref(p), None) == ttie.TTIE_ERR_INVALID
    p = ttie.default_params(tc_scale=-1.0)
    assert lib.ttie_create(ctypes.byref(h), ctypes.byref(p), None) == ttie.TTIE_ERR_INVALID
    p = ttie.default_params(inst_threads=100)
    assert lib.ttie_create(ctypes.byref(h), ctypes.byref(p), None) == ttie.TTIE_ERR_INVALID
    p = ttie.default_params(test_withhold=2)
    assert lib.ttie_create(ctypes.byref(h), ctypes.byref(p), None) == ttie.TTIE_ERR_INVALID
    p = ttie.default_params(pcg_precond=3)
    assert lib.ttie_create(ctypes.byref(h), ctypes.byref(p), None) == ttie.TTIE_ERR_INVALID
    for deg in (-1, 9):
        p = ttie.default_params(pcg_precond=ttie.PCG_CHEBYSHEV, pcg_cheb_degree=deg)
        assert lib.ttie_create(ctypes.byref(h), ctypes.byref(p), None) == ttie.TTIE_ERR_INVALID
    p = ttie.default_params(ls_rule=2)
    assert lib.ttie_create(ctypes.byref(h), ctypes.byref(p), None) == ttie.TTIE_ERR_INVALID
    p = ttie.default_params(push_eta_max=-1.0)
    assert lib.ttie_create(ctypes.byref(h), ctypes.byref(p), None) == ttie.TTIE_ERR_INVALID
    p = ttie.default_params(pcg_kernel=4)
    assert lib.ttie_create(ctypes.byref(h), ctypes.byref(p), None) == ttie.TTIE_ERR_INVALID
    p = ttie.default_params(exact_only=3)
    assert lib.ttie_create(ctypes.byref(h), ctypes.byref(p), None) == ttie.TTIE_ERR_INVALID
    p = ttie.default_params(traversal_mode=2)
    assert lib.ttie_create(ctypes.byref(h), ctypes.byref(p), None) == ttie.TTIE_ERR_INVALID


def test_no_device_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2606_06511_gb300 import ttie
    h = ctypes.c_void_p()
    p = ttie.default_params()
    assert lib.ttie_create(ctypes.byref(h), ctypes.byref(p), None) == ttie.TTIE_ERR_CUDA


def test_struct_layouts_match_the_library(lib):
    """The binding's ctypes structs have the sizes of the C structs of this build (a field
    missing, added or reordered in one of them changes a size or an offset)."""
    from paper_2606_06511_gb300 import ttie
    out = (ctypes.c_int64 * 5)()
    lib.ttie_struct_sizes(out)
    assert list(out) == [ctypes.sizeof(ttie.Params), ctypes.sizeof(ttie.BsrView), ctypes.sizeof(ttie.StepInfo),
                         ctypes.sizeof(ttie.Elastic), ctypes.sizeof(ttie.SolveInfo)]
