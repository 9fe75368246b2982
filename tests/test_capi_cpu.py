"""The C-ABI library builds, loads without a GPU and exports every function
that include/gnk.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gnk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gnk_[a-z_A-Z0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1308_5351_gb300 import build, gnk
    build.build()
    return gnk.load()


def test_header_declares_the_boundary_calls():
    names = _declared()
    for required in ("gnk_build_boundary", "gnk_apply_IminusN", "gnk_apply_M", "gnk_apply_adjoint",
                     "gnk_solve_ie", "gnk_solve_adjoint_ie", "gnk_compute_h"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_1308_5351_gb300 import gnk
    assert set(gnk.EXPORTED) == set(_declared())


def test_host_only_calls(lib):
    from paper_1308_5351_gb300 import gnk
    o = gnk.gnk_default_options()
    assert o.restart == 20 and o.maxit == 50 and abs(o.tol - 1e-12) < 1e-30
    assert o.precision == gnk.GNK_PREC_FP64
    assert "sm_103a" in gnk.gnk_version()


def test_argument_errors_before_any_launch(lib):
    """Bad sizes and NULL pointers are rejected on the host (no CUDA call)."""
    from paper_1308_5351_gb300 import gnk
    h = ctypes.c_void_p()
    buf = (ctypes.c_double * 64)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    assert lib.gnk_build_boundary(ctypes.byref(h), 2, 7, p, p, None, p, None, 1, None) == gnk.GNK_EINVAL
    assert "n even" in gnk.last_error()
    assert lib.gnk_build_boundary(ctypes.byref(h), 0, 8, p, p, None, p, None, 1, None) == gnk.GNK_EINVAL
    assert lib.gnk_build_boundary(ctypes.byref(h), 2, 8, None, p, None, p, None, 1, None) == gnk.GNK_EINVAL
    assert lib.gnk_apply_IminusN(None, p, p, 0, None) == gnk.GNK_EINVAL
    assert lib.gnk_free_boundary(None) == gnk.GNK_OK
    # the slit maps' adjoint route: NULL arrays, odd n and a NULL handle
    assert lib.gnk_slit_map_adjoint_data(2, 8, None, p, 1, p, None) == gnk.GNK_EINVAL
    assert lib.gnk_slit_map_adjoint_data(2, 7, p, p, 1, p, None) == gnk.GNK_EINVAL
    assert lib.gnk_slit_map_adjoint(None, p, p, None, p, None, None, None, None, None) == gnk.GNK_EINVAL
    assert lib.gnk_slit_map_adjoint_eval(None, p, p, 4, p, p, 0, None) == gnk.GNK_EINVAL


def test_binding_refuses_missing_library(tmp_path):
    """No fallback: a missing library is an error, not a silent CPU path."""
    from paper_1308_5351_gb300 import gnk
    old = gnk._lib
    try:
        gnk._lib = None
        with pytest.raises(RuntimeError):
            gnk.load(str(tmp_path / "missing.so"))
    finally:
        gnk._lib = old


def test_noalloc_binding_rejects_bad_operands_before_any_call(monkeypatch):
    """The binding of gnk_cauchy_sum_noalloc refuses arrays that hold fewer
    than N complex values, wrong dtypes and non-CUDA memory before it touches
    the library (which cannot see the arrays' lengths)."""
    torch = pytest.importorskip("torch")
    from paper_1308_5351_gb300 import gnk

    def no_library(*a, **k):
        raise AssertionError("the library must not be called")
    monkeypatch.setattr(gnk, "load", no_library)
    N = 16
    full = torch.zeros(N, dtype=torch.complex128)
    cases = [
        (torch.zeros(N - 1, dtype=torch.complex128), "fewer than N"),
        (torch.zeros(2 * N - 2, dtype=torch.float64), "fewer than N"),  # float64 pairs: 15 values
        (torch.zeros(N, dtype=torch.complex64), "dtype"),
        (full, "not on the current CUDA device" if torch.cuda.is_available() else "current CUDA device"),
    ]
    for bad, msg in cases:
        for pos in range(3):
            args = [full, full, full]
            args[pos] = bad
            with pytest.raises(gnk.GnkError) as e:
                gnk.gnk_cauchy_sum_noalloc(N, *args)
            assert e.value.code == gnk.GNK_EINVAL and msg in str(e.value), (pos, str(e.value))
    with pytest.raises(gnk.GnkError) as e:
        gnk.gnk_cauchy_sum_noalloc(N, full.numpy(), full, full)
    assert "must be a CUDA tensor" in str(e.value)
