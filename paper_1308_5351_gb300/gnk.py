"""Python binding of the C ABI of libgnk (include/gnk.h).

Argument marshalling only: every function below passes pointers and sizes to
the function of the same name in libgnk.so; all arithmetic runs in the CUDA
library.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays: real
arrays are float64, complex arrays complex128 (or float64 with a trailing
dimension of 2).  The library loads from this package's _lib/ directory and
raises if it has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

try:  # torch is plumbing only: device memory and streams
    import torch
except Exception:  # pragma: no cover
    torch = None

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgnk.so")

GNK_OK = 0
GNK_EINVAL = -1
GNK_ENOTCONV = -2
GNK_ENONFINITE = -3
GNK_ECUDA = -4
GNK_ENOMEM = -5

GNK_PREC_FP64 = 0
GNK_PREC_MIXED = 1
GNK_PREC_FP32 = 2
GNK_PREC_DF32 = 3
GNK_PREC_MIXED_DF = 4
GNK_PREC_FMM = 5
GNK_PREC_MIXED_FMM = 6
GNK_BUILD_DEFER = 0x100
GNK_BUILD_PLAIN = 0x200

EXPORTED = (
    "gnk_default_options", "gnk_last_error", "gnk_version", "gnk_build_boundary",
    "gnk_free_boundary", "gnk_boundary_size", "gnk_cauchy_sum", "gnk_apply_IminusN",
    "gnk_apply_M", "gnk_apply_circulant", "gnk_apply_adjoint", "gnk_solve_ie",
    "gnk_compute_h", "gnk_solve_adjoint_ie", "gnk_kernel_launches", "gnk_profile_enable",
    "gnk_profile_query", "gnk_profile_query_ex", "gnk_cauchy_sum_noalloc", "gnk_build_boundary_ex", "gnk_fbie",
    "gnk_solve_ie_transpose", "gnk_fbie_backward", "gnk_build_batch", "gnk_free_batch",
    "gnk_batch_sizes", "gnk_batch_tuning", "gnk_batch_fbie", "gnk_batch_apply_IminusN",
    "gnk_cauchy_eval", "gnk_slit_map_data", "gnk_slit_map", "gnk_slit_map_eval", "gnk_profile_mask",
    "gnk_debug_recip_f64", "gnk_debug_split_f64", "gnk_debug_barrier_fault", "gnk_profile_query_bytes",
    "gnk_slit_map_adjoint_data", "gnk_slit_map_adjoint", "gnk_slit_map_adjoint_eval",
)

PROF_PAIR64, PROF_PAIR32, PROF_REDUCE, PROF_CIRC, PROF_KRYLOV, PROF_OTHER, PROF_PAIRDF, PROF_FMM, \
    PROF_FMMNEAR, PROF_FMML2P, PROF_FMMUP, PROF_FMML2L = range(12)


class gnk_options(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("maxit", ctypes.c_int), ("tol", ctypes.c_double),
                ("precision", ctypes.c_int), ("max_refine", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("tile_chunks", ctypes.c_int),
                ("tile_variant", ctypes.c_int), ("timing", ctypes.c_int)]


class gnk_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("cycles", ctypes.c_int),
                ("refinements", ctypes.c_int), ("matvecs_fp64", ctypes.c_int),
                ("matvecs_fp32", ctypes.c_int), ("relres", ctypes.c_double),
                ("setup_ms", ctypes.c_double), ("rhs_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("h_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GnkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libgnk error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libgnk.so (built by paper_1308_5351_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(python paper_1308_5351_gb300/build.py)")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    lib.gnk_default_options.argtypes = [ctypes.POINTER(gnk_options)]
    lib.gnk_default_options.restype = None
    lib.gnk_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    lib.gnk_last_error.restype = I
    lib.gnk_version.argtypes = []
    lib.gnk_version.restype = ctypes.c_char_p
    lib.gnk_build_boundary.argtypes = [ctypes.POINTER(P), I, I, P, P, P, P, P, I, P]
    lib.gnk_build_boundary_ex.argtypes = [ctypes.POINTER(P), I, I, P, P, P, P, P, I, I, P]
    lib.gnk_fbie.argtypes = [P, P, P, P, P, ctypes.POINTER(gnk_options), ctypes.POINTER(gnk_result), P]
    lib.gnk_free_boundary.argtypes = [P]
    lib.gnk_boundary_size.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.gnk_cauchy_sum.argtypes = [P, P, P, I, P]
    for name in ("gnk_apply_IminusN", "gnk_apply_M", "gnk_apply_adjoint"):
        getattr(lib, name).argtypes = [P, P, P, I, P]
    lib.gnk_apply_circulant.argtypes = [P, P, P, P]
    for name in ("gnk_solve_ie", "gnk_solve_adjoint_ie"):
        getattr(lib, name).argtypes = [P, P, P, ctypes.POINTER(gnk_options),
                                       ctypes.POINTER(gnk_result), P]
    lib.gnk_compute_h.argtypes = [P, P, P, P, P, P]
    lib.gnk_profile_enable.argtypes = [I]
    lib.gnk_profile_mask.argtypes = [ctypes.c_uint]
    lib.gnk_profile_query.argtypes = [I, ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.gnk_cauchy_sum_noalloc.argtypes = [I, P, P, P, P]
    IP = ctypes.POINTER(I)
    lib.gnk_build_batch.argtypes = [ctypes.POINTER(P), I, IP, IP, IP, IP, P, P, P, I, P]
    lib.gnk_free_batch.argtypes = [P]
    lib.gnk_batch_apply_IminusN.argtypes = [P, P, P, I, P]
    lib.gnk_batch_sizes.argtypes = [P, ctypes.POINTER(ctypes.c_longlong), IP, IP]
    lib.gnk_batch_tuning.argtypes = [P, IP, IP, IP, IP, ctypes.POINTER(ctypes.c_float)]
    lib.gnk_batch_fbie.argtypes = [P, P, P, P, P, ctypes.POINTER(gnk_options),
                                   ctypes.POINTER(gnk_result), P, P]
    lib.gnk_solve_ie_transpose.argtypes = [P, P, P, ctypes.POINTER(gnk_options),
                                           ctypes.POINTER(gnk_result), P]
    lib.gnk_fbie_backward.argtypes = [P, P, P, P, P, P, P, P, P, P, ctypes.POINTER(gnk_options),
                                      ctypes.POINTER(gnk_result), P]
    lib.gnk_profile_query_ex.argtypes = [I, ctypes.POINTER(ctypes.c_longlong),
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]
    lib.gnk_profile_query_bytes.argtypes = [I, ctypes.POINTER(ctypes.c_longlong),
                                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.gnk_cauchy_eval.argtypes = [P, I, P, P, P, P, I, P]
    lib.gnk_slit_map_data.argtypes = [I, I, P, P, P, I, P, P, P]
    lib.gnk_slit_map.argtypes = [P, P, P, P, P, P, P, P]
    lib.gnk_slit_map_eval.argtypes = [P, P, P, P, P, P, I, P, P, I, P]
    lib.gnk_slit_map_adjoint_data.argtypes = [I, I, P, P, I, P, P]
    lib.gnk_slit_map_adjoint.argtypes = [P, P, P, ctypes.POINTER(gnk_options), P, P, P, P,
                                         ctypes.POINTER(gnk_result), P]
    lib.gnk_slit_map_adjoint_eval.argtypes = [P, P, P, I, P, P, I, P]
    lib.gnk_debug_recip_f64.argtypes = [I, P, P, P, P]
    lib.gnk_debug_split_f64.argtypes = [I, P, P, P, P]
    lib.gnk_debug_barrier_fault.argtypes = [I, I]
    lib.gnk_kernel_launches.argtypes = []
    lib.gnk_kernel_launches.restype = ctypes.c_ulonglong
    _lib = lib
    return lib


def last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    load().gnk_last_error(buf, len(buf))
    return buf.value.decode()


def _check(code, ok=(GNK_OK,)):
    if code not in ok:
        raise GnkError(code, last_error())
    return code


# --------------------------------------------------------------- marshalling
def _ptr(a, complex_: bool = False):
    """Pointer to the data of a contiguous float64 / complex128 array."""
    if a is None:
        return None
    if torch is not None and isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        ok = (torch.complex128,) if complex_ else (torch.float64,)
        if a.dtype not in ok + ((torch.float64,) if complex_ else ()):
            raise TypeError(f"expected {ok[0]}, got {a.dtype}")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        ok = (np.complex128, np.float64) if complex_ else (np.float64,)
        if a.dtype.type not in ok:
            raise TypeError(f"expected {ok[0]}, got {a.dtype}")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream):
    if stream is None:
        if torch is not None and torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return None
    if torch is not None and isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _like(a, shape, dtype_np, dtype_t):
    if torch is not None and isinstance(a, torch.Tensor):
        return torch.empty(shape, dtype=dtype_t, device=a.device)
    return np.empty(shape, dtype=dtype_np)


def _real_like(a, n):
    return _like(a, (n,), np.float64, torch.float64 if torch is not None else None)


# --------------------------------------------------------------- C-ABI mirrors
def gnk_default_options() -> gnk_options:
    o = gnk_options()
    load().gnk_default_options(ctypes.byref(o))
    return o


def gnk_kernel_launches() -> int:
    return int(load().gnk_kernel_launches())


def gnk_profile_enable(on: bool):
    return _check(load().gnk_profile_enable(1 if on else 0))


def gnk_profile_mask(mask: int):
    return _check(load().gnk_profile_mask(int(mask) & 0xffffffff))


def gnk_profile_query(kind: int):
    """(launches, total device ms, total work) of one instrumented kernel kind."""
    n, ms, wk = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
    _check(load().gnk_profile_query(int(kind), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(wk)))
    return n.value, ms.value, wk.value


def gnk_profile_query_ex(kind: int):
    """(launches, total device ms, total work, algorithmic pipe instructions)."""
    n, ms, wk, ins = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().gnk_profile_query_ex(int(kind), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(wk),
                                       ctypes.byref(ins)))
    return n.value, ms.value, wk.value, ins.value


def gnk_profile_query_bytes(kind: int):
    """(launches, total device ms, total work, pipe instructions, algorithmic bytes)."""
    n, ms, wk, ins, by = (ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double(),
                          ctypes.c_double())
    _check(load().gnk_profile_query_bytes(int(kind), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(wk),
                                          ctypes.byref(ins), ctypes.byref(by)))
    return n.value, ms.value, wk.value, ins.value, by.value


def gnk_version() -> str:
    return load().gnk_version().decode()


def gnk_build_boundary(m1, n, et, etp, A, etpp=None, Ap=None, bounded=True, stream=None):
    """Returns an opaque handle (ctypes.c_void_p)."""
    h = ctypes.c_void_p()
    _check(load().gnk_build_boundary(ctypes.byref(h), int(m1), int(n), _ptr(et, True),
                                     _ptr(etp, True), _ptr(etpp, True), _ptr(A, True),
                                     _ptr(Ap, True), 1 if bounded else 0, _stream(stream)))
    return h


def gnk_build_boundary_ex(m1, n, et, etp, A, etpp=None, Ap=None, bounded=True,
                          precision=GNK_PREC_FP64, stream=None):
    h = ctypes.c_void_p()
    _check(load().gnk_build_boundary_ex(ctypes.byref(h), int(m1), int(n), _ptr(et, True),
                                        _ptr(etp, True), _ptr(etpp, True), _ptr(A, True),
                                        _ptr(Ap, True), 1 if bounded else 0, int(precision),
                                        _stream(stream)))
    return h


def gnk_fbie(h, gam, mu, hv, hk=None, options: Optional[gnk_options] = None, stream=None):
    res = gnk_result()
    code = load().gnk_fbie(h, _ptr(gam), _ptr(mu), _ptr(hv), _ptr(hk),
                           ctypes.byref(options) if options is not None else None,
                           ctypes.byref(res), _stream(stream))
    _check(code, (GNK_OK, GNK_ENOTCONV))
    return res


def gnk_free_boundary(h):
    return _check(load().gnk_free_boundary(h))


def gnk_boundary_size(h):
    m1, n = ctypes.c_int(), ctypes.c_int()
    _check(load().gnk_boundary_size(h, ctypes.byref(m1), ctypes.byref(n)))
    return m1.value, n.value


def gnk_cauchy_sum(h, w, z, precision=GNK_PREC_FP64, stream=None):
    return _check(load().gnk_cauchy_sum(h, _ptr(w, True), _ptr(z, True), int(precision),
                                        _stream(stream)))


def _noalloc_operand(name, a, N):
    """Checks one array of gnk_cauchy_sum_noalloc before any launch: a
    contiguous complex128 (or float64 pairs) CUDA tensor on the current device
    holding at least N complex values."""
    if torch is None or not isinstance(a, torch.Tensor):
        raise GnkError(GNK_EINVAL, f"gnk_cauchy_sum_noalloc: {name} must be a CUDA tensor "
                                   "(nothing is staged or copied)")
    if a.dtype == torch.complex128:
        held = a.numel()
    elif a.dtype == torch.float64:
        held = a.numel() // 2
    else:
        raise GnkError(GNK_EINVAL, f"gnk_cauchy_sum_noalloc: {name} has dtype {a.dtype}; "
                                   "expected complex128 or float64 (re, im) pairs")
    if held < N:
        raise GnkError(GNK_EINVAL, f"gnk_cauchy_sum_noalloc: {name} holds {held} complex values, "
                                   f"fewer than N = {N}")
    if not a.is_contiguous():
        raise GnkError(GNK_EINVAL, f"gnk_cauchy_sum_noalloc: {name} must be contiguous")


def _noalloc_device(name, a):
    if not a.is_cuda or a.device.index != torch.cuda.current_device():
        raise GnkError(GNK_EINVAL, f"gnk_cauchy_sum_noalloc: {name} is on {a.device}, not on the "
                                   "current CUDA device")


def gnk_cauchy_sum_noalloc(N, et, w, z, stream=None):
    """z = E w with no device allocation: et, w, z CUDA tensors on the current
    device holding at least N complex values each, N <= 65536."""
    N = int(N)
    ops = (("et", et), ("w", w), ("z", z))
    for name, a in ops:
        _noalloc_operand(name, a, N)
    for name, a in ops:
        _noalloc_device(name, a)
    return _check(load().gnk_cauchy_sum_noalloc(N, _ptr(et, True), _ptr(w, True),
                                                _ptr(z, True), _stream(stream)))


def gnk_debug_recip_f64(x, y_lib, y_div, stream=None):
    """The pair kernels' FP64 reciprocal and CUDA's 1.0/x of the device array x."""
    n = int(x.numel())
    for a in (y_lib, y_div):
        if a.numel() < n:
            raise GnkError(GNK_EINVAL, "gnk_debug_recip_f64: output shorter than x")
    return _check(load().gnk_debug_recip_f64(n, _ptr(x), _ptr(y_lib), _ptr(y_div), _stream(stream)))


def gnk_debug_split_f64(x, hi, lo, stream=None):
    """The FMM kernels' bit-level double-float split (hi, lo float32) of the device array x."""
    n = int(x.numel())
    for a in (hi, lo):
        if a.numel() < n:
            raise GnkError(GNK_EINVAL, "gnk_debug_split_f64: output shorter than x")
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise GnkError(GNK_EINVAL, "gnk_debug_split_f64: outputs must be contiguous float32")
    return _check(load().gnk_debug_split_f64(n, _ptr(x), ctypes.c_void_p(hi.data_ptr()),
                                             ctypes.c_void_p(lo.data_ptr()), _stream(stream)))


def gnk_debug_barrier_fault(skip_block: int, spin_limit: int = 0):
    """Test hook: block `skip_block` of later Arnoldi steps skips its grid-barrier
    arrivals (-1: none); the other blocks' waits give up after spin_limit polls."""
    return _check(load().gnk_debug_barrier_fault(int(skip_block), int(spin_limit)))


def gnk_cauchy_eval(h, z, f, fz, finf=None, precision=GNK_PREC_FP64, stream=None):
    """fz = f(z) at points z of G by the Cauchy integral formula (Eqs. cauchy4, cauchy6)."""
    fi = None
    if finf is not None:
        c = complex(finf)
        fi = (ctypes.c_double * 2)(c.real, c.imag)
    nz = int(z.numel() if torch is not None and isinstance(z, torch.Tensor) else z.size)
    return _check(load().gnk_cauchy_eval(h, nz, _ptr(z, True), _ptr(f, True), fi, _ptr(fz, True),
                                         int(precision), _stream(stream)))


def _c2(alpha):
    c = complex(alpha)
    return (ctypes.c_double * 2)(c.real, c.imag)


def gnk_slit_map_data(m1, n, et, alpha, theta, A, gam, stream=None, bounded=True):
    """A = e^{i(pi/2 - theta)} (eta - alpha) (bounded G) or e^{i(pi/2 - theta)}
    (unbounded G), gamma = -Re[e^{i(pi/2 - theta)} log(eta - alpha)]."""
    return _check(load().gnk_slit_map_data(int(m1), int(n), _ptr(et, True), _c2(alpha), _ptr(theta),
                                           1 if bounded else 0, _ptr(A, True), _ptr(gam), _stream(stream)))


def gnk_slit_map(h, alpha, gam, mu, hv, hk, w, stream=None):
    """w at the nodes of the slit map (Sec. 7, Ex. 3)."""
    return _check(load().gnk_slit_map(h, _c2(alpha), _ptr(gam), _ptr(mu), _ptr(hv), _ptr(hk), _ptr(w, True),
                                      _stream(stream)))


def gnk_slit_map_eval(h, alpha, gam, mu, hv, hk, z, wz, precision=GNK_PREC_FP64, stream=None):
    """w at points z of G (Cauchy formula for f)."""
    nz = int(z.numel() if torch is not None and isinstance(z, torch.Tensor) else z.size)
    return _check(load().gnk_slit_map_eval(h, _c2(alpha), _ptr(gam), _ptr(mu), _ptr(hv), _ptr(hk), nz,
                                           _ptr(z, True), _ptr(wz, True), int(precision), _stream(stream)))


def slit_map(dom, alpha, theta, z=None, device="cuda", precision=GNK_PREC_FMM, tol=1e-12, stream=None):
    """The slit map of a domain (curves, n and boundedness of `dom`): returns
    (w at the nodes, h_k, w at z or None, gnk_result).  theta: one value per
    boundary (pi/2 circular slit, 0 radial slit).  Cauchy sums by `precision`
    (GNK_PREC_FMM by default; GNK_PREC_FP64 or _DF32 direct)."""
    et = torch.as_tensor(np.ascontiguousarray(dom.et), device=device)
    etp = torch.as_tensor(np.ascontiguousarray(dom.etp), device=device)
    th = torch.as_tensor(np.asarray(theta, dtype=np.float64), device=device)
    A = torch.empty_like(et)
    gam = torch.empty(dom.N, dtype=torch.float64, device=device)
    gnk_slit_map_data(dom.m1, dom.n, et, alpha, th, A, gam, stream, bounded=dom.bounded)
    bprec = GNK_PREC_FMM if precision == GNK_PREC_FMM else GNK_PREC_FP64
    with Boundary(dom.m1, dom.n, et, etp, A, None, None, dom.bounded, stream, bprec) as b:
        mu, h, hk, res = b.fbie(gam, tol=tol, precision=precision, stream=stream)
        w = torch.empty_like(et)
        gnk_slit_map(b.handle, alpha, gam, mu, h, hk, w, stream)
        wz = None
        if z is not None:
            zt = torch.as_tensor(np.ascontiguousarray(z, dtype=np.complex128), device=device)
            wz = torch.empty_like(zt)
            ep = GNK_PREC_DF32 if precision in (GNK_PREC_DF32, GNK_PREC_MIXED_DF) else GNK_PREC_FP64
            gnk_slit_map_eval(b.handle, alpha, gam, mu, h, hk, zt, wz, ep, stream)
    return w, hk, wz, res


def gnk_slit_map_adjoint_data(m1, n, etp, theta, Ap, stream=None, bounded=True):
    """A' of the slit map's A (e^{i(pi/2 - theta)} eta' for bounded G, 0 for
    unbounded G), for a handle that solves Eq. (ie*)."""
    return _check(load().gnk_slit_map_adjoint_data(int(m1), int(n), _ptr(etp, True), _ptr(theta),
                                                   1 if bounded else 0, _ptr(Ap, True), _stream(stream)))


def gnk_slit_map_adjoint(h, alpha, theta, w, omega=None, psi=None, params=None,
                         options: Optional[gnk_options] = None, stream=None):
    """The slit map by solves of the adjoint equation only (Sec. 7, Ex. 3 and
    Ex. 4): w (and optionally omega, psi, params) at the nodes; returns the
    gnk_result of the solves."""
    res = gnk_result()
    code = load().gnk_slit_map_adjoint(h, _c2(alpha), _ptr(theta), ctypes.byref(options) if options is not None
                                       else None, _ptr(w, True), _ptr(omega, True), _ptr(psi), _ptr(params),
                                       ctypes.byref(res), _stream(stream))
    _check(code, (GNK_OK, GNK_ENOTCONV))
    return res


def gnk_slit_map_adjoint_eval(h, alpha, omega, z, wz, precision=GNK_PREC_FP64, stream=None):
    """w at points z of G from omega at the nodes (Cauchy formula for omega)."""
    nz = int(z.numel() if torch is not None and isinstance(z, torch.Tensor) else z.size)
    return _check(load().gnk_slit_map_adjoint_eval(h, _c2(alpha), _ptr(omega, True), nz, _ptr(z, True),
                                                   _ptr(wz, True), int(precision), _stream(stream)))


def slit_map_adjoint(dom, alpha, theta, z=None, device="cuda", precision=GNK_PREC_FMM, tol=1e-12,
                     restart=20, maxit=50, stream=None):
    """The slit map of a domain by the adjoint route: returns (w at the nodes,
    psi, params, omega at the nodes, w at z or None, gnk_result).  theta: one
    value per boundary (pi/2 circular slit, 0 radial slit).  Cauchy sums by
    `precision` (GNK_PREC_FMM by default)."""
    et = torch.as_tensor(np.ascontiguousarray(dom.et), device=device)
    etp = torch.as_tensor(np.ascontiguousarray(dom.etp), device=device)
    etpp = torch.as_tensor(np.ascontiguousarray(dom.etpp), device=device)
    th = torch.as_tensor(np.asarray(theta, dtype=np.float64), device=device)
    A = torch.empty_like(et)
    Ap = torch.empty_like(et)
    gam = torch.empty(dom.N, dtype=torch.float64, device=device)
    gnk_slit_map_data(dom.m1, dom.n, et, alpha, th, A, gam, stream, bounded=dom.bounded)
    gnk_slit_map_adjoint_data(dom.m1, dom.n, etp, th, Ap, stream, bounded=dom.bounded)
    bprec = GNK_PREC_FMM if precision in (GNK_PREC_FMM, GNK_PREC_MIXED_FMM) else GNK_PREC_FP64
    with Boundary(dom.m1, dom.n, et, etp, A, etpp, Ap, dom.bounded, stream, bprec) as b:
        w = torch.empty_like(et)
        omega = torch.empty_like(et)
        psi = torch.empty(dom.N, dtype=torch.float64, device=device)
        params = torch.empty(dom.m1 + 1, dtype=torch.float64, device=device)
        res = gnk_slit_map_adjoint(b.handle, alpha, th, w, omega, psi, params,
                                   options(tol=tol, precision=precision, restart=restart, maxit=maxit), stream)
        wz = None
        if z is not None:
            zt = torch.as_tensor(np.ascontiguousarray(z, dtype=np.complex128), device=device)
            wz = torch.empty_like(zt)
            ep = GNK_PREC_DF32 if precision in (GNK_PREC_DF32, GNK_PREC_MIXED_DF) else GNK_PREC_FP64
            gnk_slit_map_adjoint_eval(b.handle, alpha, omega, zt, wz, ep, stream)
    return w, psi, params, omega, wz, res


def gnk_apply_IminusN(h, x, y, precision=GNK_PREC_FP64, stream=None):
    return _check(load().gnk_apply_IminusN(h, _ptr(x), _ptr(y), int(precision), _stream(stream)))


def gnk_apply_M(h, x, y, precision=GNK_PREC_FP64, stream=None):
    return _check(load().gnk_apply_M(h, _ptr(x), _ptr(y), int(precision), _stream(stream)))


def gnk_apply_adjoint(h, x, y, precision=GNK_PREC_FP64, stream=None):
    return _check(load().gnk_apply_adjoint(h, _ptr(x), _ptr(y), int(precision), _stream(stream)))


def gnk_apply_circulant(h, x, y, stream=None):
    return _check(load().gnk_apply_circulant(h, _ptr(x), _ptr(y), _stream(stream)))


def gnk_solve_ie(h, gam, mu, options: Optional[gnk_options] = None, stream=None):
    res = gnk_result()
    code = load().gnk_solve_ie(h, _ptr(gam), _ptr(mu),
                               ctypes.byref(options) if options is not None else None,
                               ctypes.byref(res), _stream(stream))
    _check(code, (GNK_OK, GNK_ENOTCONV))
    return res


def gnk_solve_adjoint_ie(h, gam, mu, options: Optional[gnk_options] = None, stream=None):
    res = gnk_result()
    code = load().gnk_solve_adjoint_ie(h, _ptr(gam), _ptr(mu),
                                       ctypes.byref(options) if options is not None else None,
                                       ctypes.byref(res), _stream(stream))
    _check(code, (GNK_OK, GNK_ENOTCONV))
    return res


def gnk_solve_ie_transpose(h, rhs, x, options: Optional[gnk_options] = None, stream=None):
    res = gnk_result()
    code = load().gnk_solve_ie_transpose(h, _ptr(rhs), _ptr(x),
                                         ctypes.byref(options) if options is not None else None,
                                         ctypes.byref(res), _stream(stream))
    _check(code, (GNK_OK, GNK_ENOTCONV))
    return res


def gnk_fbie_backward(h, mu, gam, grad_mu, grad_h, grad_et, grad_etp, grad_A, grad_gam,
                      options: Optional[gnk_options] = None, stream=None, grad_hk=None):
    """grad_hk (nullable, m1 values): dL/dh_k of the component means."""
    res = gnk_result()
    code = load().gnk_fbie_backward(h, _ptr(mu), _ptr(gam), _ptr(grad_mu), _ptr(grad_h), _ptr(grad_hk),
                                    _ptr(grad_et, True), _ptr(grad_etp, True), _ptr(grad_A, True),
                                    _ptr(grad_gam),
                                    ctypes.byref(options) if options is not None else None,
                                    ctypes.byref(res), _stream(stream))
    _check(code, (GNK_OK, GNK_ENOTCONV))
    return res


def gnk_compute_h(h, mu, gam, hv, hk=None, stream=None):
    return _check(load().gnk_compute_h(h, _ptr(mu), _ptr(gam), _ptr(hv), _ptr(hk),
                                       _stream(stream)))


def options(**kw) -> gnk_options:
    o = gnk_default_options()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


# --------------------------------------------------------------- convenience
class Boundary:
    """Owns one gnk_boundary handle built from a domain's arrays (numpy complex
    arrays on the host, or complex128 CUDA tensors)."""

    def __init__(self, m1, n, et, etp, A, etpp=None, Ap=None, bounded=True, stream=None,
                 precision=GNK_PREC_FP64):
        self.m1, self.n, self.N = int(m1), int(n), int(m1) * int(n)
        self.handle = None
        self.handle = gnk_build_boundary_ex(m1, n, et, etp, A, etpp, Ap, bounded, precision, stream)

    @classmethod
    def from_domain(cls, dom, adjoint=True, device=None, stream=None, precision=GNK_PREC_FP64,
                    plain=False):
        """plain=True: the discretisation without singularity subtraction (needs
        eta'', so adjoint is implied)."""
        if plain:
            adjoint = True
            precision |= GNK_BUILD_PLAIN
        arrs = [dom.et, dom.etp, dom.A, dom.etpp if adjoint else None, dom.Ap if adjoint else None]
        if device is not None:
            arrs = [None if a is None else torch.as_tensor(np.ascontiguousarray(a), device=device)
                    for a in arrs]
        return cls(dom.m1, dom.n, arrs[0], arrs[1], arrs[2], arrs[3], arrs[4], dom.bounded, stream,
                   precision)

    def close(self):
        if self.handle is not None:
            gnk_free_boundary(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def cauchy_sum(self, w, precision=GNK_PREC_FP64, out=None, stream=None):
        z = out if out is not None else _like(w, tuple(w.shape), np.complex128,
                                              torch.complex128 if torch is not None else None)
        gnk_cauchy_sum(self.handle, w, z, precision, stream)
        return z

    def cauchy_eval(self, z, f_nodes, finf=None, precision=GNK_PREC_FP64, out=None, stream=None):
        """f at the points z of G from its boundary values f_nodes (complex, N)."""
        fz = out if out is not None else _like(z, tuple(z.shape), np.complex128,
                                               torch.complex128 if torch is not None else None)
        gnk_cauchy_eval(self.handle, z, f_nodes, fz, finf, precision, stream)
        return fz

    def _unary(self, fn, x, precision, out, stream):
        y = out if out is not None else _real_like(x, self.N)
        if precision is None:
            fn(self.handle, x, y, stream=stream)
        else:
            fn(self.handle, x, y, precision, stream)
        return y

    def apply_IminusN(self, x, precision=GNK_PREC_FP64, out=None, stream=None):
        return self._unary(gnk_apply_IminusN, x, precision, out, stream)

    def apply_M(self, x, precision=GNK_PREC_FP64, out=None, stream=None):
        return self._unary(gnk_apply_M, x, precision, out, stream)

    def apply_adjoint(self, x, precision=GNK_PREC_FP64, out=None, stream=None):
        return self._unary(gnk_apply_adjoint, x, precision, out, stream)

    def apply_circulant(self, x, out=None, stream=None):
        return self._unary(gnk_apply_circulant, x, None, out, stream)

    def solve_ie(self, gam, out=None, stream=None, **opts):
        mu = out if out is not None else _real_like(gam, self.N)
        res = gnk_solve_ie(self.handle, gam, mu, options(**opts), stream)
        return mu, res

    def solve_adjoint_ie(self, gam, out=None, stream=None, **opts):
        mu = out if out is not None else _real_like(gam, self.N)
        res = gnk_solve_adjoint_ie(self.handle, gam, mu, options(**opts), stream)
        return mu, res

    def fbie(self, gam, stream=None, **opts):
        """(mu, h, h_k, result) of the FBIE computation in one call."""
        mu = _real_like(gam, self.N)
        h = _real_like(gam, self.N)
        hk = _real_like(gam, self.m1)
        res = gnk_fbie(self.handle, gam, mu, h, hk, options(**opts), stream)
        return mu, h, hk, res

    def compute_h(self, mu, gam, out=None, hk=None, stream=None):
        h = out if out is not None else _real_like(mu, self.N)
        hk = hk if hk is not None else _real_like(mu, self.m1)
        gnk_compute_h(self.handle, mu, gam, h, hk, stream)
        return h, hk


# --------------------------------------------------------------- batches
def _ints(v):
    arr = (ctypes.c_int * len(v))(*[int(x) for x in v])
    return arr


class Batch:
    """Owns one gnk_batch: domains given as lists of Domain-like objects
    (numpy complex arrays et, etp, A) with a right-hand-side count each."""

    def __init__(self, domains, nrhs, autotune=True, device=None, stream=None):
        self.m1 = [d.m1 for d in domains]
        self.n = [d.n for d in domains]
        self.nrhs = [int(r) for r in nrhs]
        bounded = [1 if d.bounded else 0 for d in domains]
        arrs = [np.ascontiguousarray(np.concatenate([getattr(d, k) for d in domains]))
                for k in ("et", "etp", "A")]
        if device is not None:
            arrs = [torch.as_tensor(a, device=device) for a in arrs]
        h = ctypes.c_void_p()
        self.handle = None
        _check(load().gnk_build_batch(ctypes.byref(h), len(domains), _ints(self.m1), _ints(self.n),
                                      _ints(self.nrhs), _ints(bounded), _ptr(arrs[0], True),
                                      _ptr(arrs[1], True), _ptr(arrs[2], True), 1 if autotune else 0,
                                      _stream(stream)))
        self.handle = h
        L, ns, nhk = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int()
        _check(load().gnk_batch_sizes(h, ctypes.byref(L), ctypes.byref(ns), ctypes.byref(nhk)))
        self.L, self.nsys, self.nhk = L.value, ns.value, nhk.value

    def tuning(self):
        v = [ctypes.c_int() for _ in range(4)]
        ms = (ctypes.c_float * 7)()
        _check(load().gnk_batch_tuning(self.handle, *[ctypes.byref(x) for x in v], ms))
        return {"fp32_targets": v[0].value, "fp32_group": v[1].value, "df_targets": v[2].value,
                "df_group": v[3].value, "variant_ms": list(ms)}

    def fbie(self, gam, stream=None, **opts):
        o = options(precision=GNK_PREC_MIXED_DF)
        for k, v in opts.items():
            setattr(o, k, v)
        mu = _real_like(gam, self.L)
        h = _real_like(gam, self.L)
        hk = _real_like(gam, self.nhk)
        rel = np.zeros(self.nsys)
        res = gnk_result()
        code = load().gnk_batch_fbie(self.handle, _ptr(gam), _ptr(mu), _ptr(h), _ptr(hk),
                                     ctypes.byref(o), ctypes.byref(res),
                                     ctypes.c_void_p(rel.ctypes.data), _stream(stream))
        _check(code, (GNK_OK, GNK_ENOTCONV))
        return mu, h, hk, res, rel

    def apply_IminusN(self, x, precision=GNK_PREC_FP32, stream=None):
        y = _real_like(x, self.L)
        _check(load().gnk_batch_apply_IminusN(self.handle, _ptr(x), _ptr(y), int(precision),
                                              _stream(stream)))
        return y

    def close(self):
        if self.handle is not None:
            load().gnk_free_batch(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
