"""ctypes binding of libairga.so (C ABI in include/airga.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  PyTorch supplies device memory (tensors) and the current stream.
Function names follow the C entry points without the ``airga_`` prefix.

The library is loaded from this package directory; if it is missing the
import of any compute function raises instead of falling back to anything.
With AIRGA_LIB=checked in the environment the bounds-checked build
(libairga_checked.so, see build.build(checked=True)) is loaded instead.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libairga.so")
LIB_CHECKED_PATH = os.path.join(HERE, "libairga_checked.so")

OK = 0
E_INVALID_ARG, E_SHAPE, E_BREAKDOWN, E_MAXIT, E_TIMEOUT = 1, 2, 3, 4, 5
E_RANK, E_CUDA, E_OOM, E_UNSUPPORTED = 6, 7, 8, 9
SPAI_QR, SPAI_MR, SPAI_NE = 0, 1, 2

# every symbol include/airga.h declares
EXPORTS = (
    "airga_options_default", "airga_status_string", "airga_last_error", "airga_version",
    "airga_mat_from_csr", "airga_mat_from_band", "airga_mat_to_band", "airga_mat_rows",
    "airga_mat_free", "airga_assemble_shifted", "airga_spmv", "airga_spai_build",
    "airga_spai_update", "airga_precond_apply", "airga_precond_length", "airga_precond_rows",
    "airga_precond_factor", "airga_precond_from_bands", "airga_precond_status",
    "airga_precond_free", "airga_pcg_solve", "airga_true_residual", "airga_debug_set_fault",
    "airga_trim", "airga_pcg_solve_noalloc", "airga_pcg_solve_mixed", "airga_batch_create",
    "airga_batch_solve", "airga_batch_info", "airga_batch_free", "airga_pcg_solve_mv",
    "airga_mlp_train_options_default", "airga_mlp_create", "airga_mlp_set_params",
    "airga_mlp_get_params", "airga_mlp_status", "airga_mlp_features", "airga_mlp_forward",
    "airga_mlp_grad", "airga_mlp_train", "airga_mlp_spai", "airga_mlp_free",
    "airga_debug_force_pcg_kernel", "airga_mat_is_banded", "airga_mat_nnz", "airga_mat_to_csr",
    "airga_precond_is_banded", "airga_precond_factor_nnz", "airga_precond_factor_csr",
    "airga_precond_from_csr", "airga_probe_fp64_rate", "airga_debug_pool_used",
    "airga_debug_checked", "airga_debug_check_selftest", "airga_probe_read_bw",
    "airga_debug_record_placement", "airga_stream_hold", "airga_trace_enable", "airga_trace_read",
)

MLP_IN, MLP_HIDDEN, MLP_OUT, MLP_NPARAM = 16, 64, 16, 6288


class TraceRecord(C.Structure):
    """airga_trace_record: one traced C-ABI call."""
    _fields_ = [("name", C.c_char_p), ("ms", C.c_double), ("stream", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [
        ("tol", C.c_double),
        ("maxit", C.c_int32),
        ("spai_mode", C.c_int32),
        ("mr_tol", C.c_double),
        ("mr_kmax", C.c_int32),
        ("symmetrize", C.c_int32),
        ("pattern_hbw", C.c_int32),
        ("warm_start", C.c_int32),
        ("barrier_timeout_ms", C.c_int32),
        ("want_colres", C.c_int32),
        ("inner_tol", C.c_double),
        ("max_outer", C.c_int32),
        ("mr_relative", C.c_int32),
        ("sm_share", C.c_int32),
        ("reserved0", C.c_int32),
    ]


class MlpTrainOptions(C.Structure):
    _fields_ = [
        ("lr", C.c_float),
        ("beta1", C.c_float),
        ("beta2", C.c_float),
        ("eps", C.c_float),
        ("batch", C.c_int32),
        ("cosine_steps", C.c_int32),
        ("seed", C.c_uint64),
    ]


class AirgaError(RuntimeError):
    def __init__(self, code, where, msg):
        super().__init__("%s failed: %s (%s)" % (where, msg, status_string(code)))
        self.code = code


_lib = None


def lib_path() -> str:
    """The library this process loads: libairga.so, or the bounds-checked
    libairga_checked.so when AIRGA_LIB=checked."""
    return LIB_CHECKED_PATH if os.environ.get("AIRGA_LIB", "") == "checked" else LIB_PATH


def lib():
    """Load the library once; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError("%s is not built (run paper_1606_01216_gb300.build.build(%s))"
                           % (os.path.basename(path), "checked=True" if path == LIB_CHECKED_PATH else ""))
    L = C.CDLL(path)
    vp, dp, i64, i32 = C.c_void_p, C.c_void_p, C.c_int64, C.c_int32
    sig = {
        "airga_options_default": (None, [C.POINTER(Options)]),
        "airga_status_string": (C.c_char_p, [C.c_int]),
        "airga_last_error": (C.c_char_p, []),
        "airga_version": (C.c_int, []),
        "airga_mat_from_csr": (C.c_int, [i64, i64, vp, vp, vp, vp, C.POINTER(vp)]),
        "airga_mat_from_band": (C.c_int, [i64, vp, vp, C.POINTER(vp)]),
        "airga_mat_to_band": (C.c_int, [vp, vp, vp]),
        "airga_mat_rows": (i64, [vp]),
        "airga_mat_free": (None, [vp]),
        "airga_assemble_shifted": (C.c_int, [vp, vp, C.c_double, C.c_double, C.c_double, vp,
                                             C.POINTER(vp)]),
        "airga_spmv": (C.c_int, [vp, vp, vp, i32, vp]),
        "airga_spai_build": (C.c_int, [vp, vp, C.POINTER(Options), vp, C.POINTER(vp)]),
        "airga_probe_fp64_rate": (C.c_int, [i64, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                            C.POINTER(C.c_double), vp]),
        "airga_mat_is_banded": (C.c_int, [vp]),
        "airga_mat_nnz": (i64, [vp]),
        "airga_mat_to_csr": (C.c_int, [vp, vp, vp, vp, vp]),
        "airga_precond_is_banded": (C.c_int, [vp]),
        "airga_precond_factor_nnz": (i64, [vp, i32]),
        "airga_precond_factor_csr": (C.c_int, [vp, i32, vp, vp, vp, vp]),
        "airga_precond_from_csr": (C.c_int, [i64, i32, C.POINTER(i64), C.POINTER(vp), C.POINTER(vp),
                                             C.POINTER(vp), vp, C.POINTER(vp)]),
        "airga_spai_update": (C.c_int, [vp, vp, vp, C.POINTER(Options), vp, C.POINTER(vp)]),
        "airga_precond_apply": (C.c_int, [vp, vp, vp, i32, vp]),
        "airga_precond_length": (i32, [vp]),
        "airga_precond_rows": (i64, [vp]),
        "airga_precond_factor": (C.c_int, [vp, i32, vp, vp]),
        "airga_precond_from_bands": (C.c_int, [i64, i32, C.POINTER(vp), vp, C.POINTER(vp)]),
        "airga_precond_status": (C.c_int, [vp, vp, vp, C.POINTER(C.c_int), vp]),
        "airga_precond_free": (None, [vp]),
        "airga_pcg_solve": (C.c_int, [vp, vp, vp, i32, C.POINTER(Options), vp, vp, vp, vp, vp,
                                      vp]),
        "airga_true_residual": (C.c_int, [vp, vp, vp, i32, vp, vp]),
        "airga_pcg_solve_mixed": (C.c_int, [vp, vp, vp, i32, C.POINTER(Options), vp, vp, vp, vp,
                                            vp, vp]),
        "airga_batch_create": (C.c_int, [i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                         C.POINTER(vp), C.POINTER(C.c_double),
                                         C.POINTER(C.c_int32), i32, C.POINTER(Options), vp, vp,
                                         vp, vp, C.POINTER(vp)]),
        "airga_batch_solve": (C.c_int, [vp, vp]),
        "airga_batch_info": (C.c_int, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32),
                                       C.POINTER(C.c_double)]),
        "airga_batch_free": (None, [vp]),
        "airga_pcg_solve_mv": (C.c_int, [vp, vp, vp, vp, C.c_double, i32, C.POINTER(Options), vp,
                                         vp, vp, vp, vp, vp]),
        "airga_debug_set_fault": (C.c_int, [C.c_int]),
        "airga_debug_pool_used": (C.c_int, [C.POINTER(i64)]),
        "airga_debug_checked": (C.c_int, [C.POINTER(i64), C.POINTER(i32), C.POINTER(i64)]),
        "airga_probe_read_bw": (C.c_int, [i64, i32, C.POINTER(C.c_double), C.POINTER(C.c_double), vp]),
        "airga_debug_check_selftest": (C.c_int, [i64, i64, i32, vp]),
        "airga_debug_force_pcg_kernel": (C.c_int, [C.c_int]),
        "airga_debug_record_placement": (C.c_int, [vp]),
        "airga_stream_hold": (C.c_int, [i32, vp]),
        "airga_trace_enable": (C.c_int, [i32]),
        "airga_trace_read": (C.c_int, [C.POINTER(TraceRecord), i32, C.POINTER(i32), C.POINTER(i64)]),
        "airga_pcg_solve_noalloc": (C.c_int, [i64, vp, vp, vp, i32, C.POINTER(Options), vp, vp,
                                              vp, vp, vp, vp]),
        "airga_trim": (C.c_int, []),
        "airga_mlp_train_options_default": (None, [C.POINTER(MlpTrainOptions)]),
        "airga_mlp_create": (C.c_int, [C.c_uint64, vp, C.POINTER(vp)]),
        "airga_mlp_set_params": (C.c_int, [vp, vp, vp]),
        "airga_mlp_get_params": (C.c_int, [vp, vp, vp]),
        "airga_mlp_status": (C.c_int, [vp, C.POINTER(i64), C.POINTER(C.c_int), vp]),
        "airga_mlp_features": (C.c_int, [vp, vp, C.c_double, C.c_double, C.c_double, vp, i64,
                                         vp, vp, vp, vp, vp]),
        "airga_mlp_forward": (C.c_int, [vp, vp, i64, vp, vp]),
        "airga_mlp_grad": (C.c_int, [vp, vp, vp, vp, i64, vp, i32, vp, vp, vp]),
        "airga_mlp_train": (C.c_int, [vp, vp, vp, vp, i64, i32, C.POINTER(MlpTrainOptions), vp,
                                      vp, vp]),
        "airga_mlp_spai": (C.c_int, [vp, vp, C.c_double, C.c_double, C.c_double, vp,
                                     C.POINTER(vp)]),
        "airga_mlp_free": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def status_string(code: int) -> str:
    return lib().airga_status_string(int(code)).decode()


def last_error() -> str:
    return lib().airga_last_error().decode()


def _check(code, where):
    if code != OK:
        raise AirgaError(code, where, last_error())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t: torch.Tensor | None, dtype=None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError("expected %s, got %s" % (dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def options(**kw) -> Options:
    o = Options()
    lib().airga_options_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


# ---------------------------------------------------------------------------
# handles
# ---------------------------------------------------------------------------

class Mat:
    """Owning wrapper of an airga_mat handle (band-7 matrix on the device)."""

    def __init__(self, handle: int, n: int):
        self.h = C.c_void_p(handle)
        self.n = int(n)

    def __del__(self):
        if getattr(self, "h", None) and self.h.value and _lib is not None:
            _lib.airga_mat_free(self.h)
            self.h = C.c_void_p(None)

    def band(self, stream=None) -> torch.Tensor:
        return mat_to_band(self, stream)


class Precond:
    """Owning wrapper of an airga_precond handle (SPAI / update chain)."""

    def __init__(self, handle: int, n: int):
        self.h = C.c_void_p(handle)
        self.n = int(n)

    def __del__(self):
        if getattr(self, "h", None) and self.h.value and _lib is not None:
            _lib.airga_precond_free(self.h)
            self.h = C.c_void_p(None)

    def __len__(self):
        return int(lib().airga_precond_length(self.h))


# ---------------------------------------------------------------------------
# matrices
# ---------------------------------------------------------------------------

def mat_from_csr(n: int, rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor,
                 stream=None) -> Mat:
    out = C.c_void_p()
    _check(lib().airga_mat_from_csr(int(n), int(col.numel()), _ptr(rowptr, torch.int64),
                                    _ptr(col, torch.int32), _ptr(val, torch.float64),
                                    _stream(stream), C.byref(out)), "mat_from_csr")
    return Mat(out.value, n)


def mat_from_band(band: torch.Tensor, stream=None) -> Mat:
    n = band.numel() // 7
    out = C.c_void_p()
    _check(lib().airga_mat_from_band(n, _ptr(band, torch.float64), _stream(stream),
                                     C.byref(out)), "mat_from_band")
    return Mat(out.value, n)


def mat_is_banded(A: Mat) -> bool:
    return bool(lib().airga_mat_is_banded(A.h))


def mat_to_csr(A: Mat, stream=None):
    """(rowptr int64, col int32, val float64) device tensors of A (rows sorted)."""
    nnz = int(lib().airga_mat_nnz(A.h))
    rp = torch.empty(A.n + 1, dtype=torch.int64, device="cuda")
    ci = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
    va = torch.empty(max(nnz, 1), dtype=torch.float64, device="cuda")
    _check(lib().airga_mat_to_csr(A.h, _ptr(rp), _ptr(ci), _ptr(va), _stream(stream)),
           "mat_to_csr")
    return rp, ci[:nnz], va[:nnz]


def mat_to_band(A: Mat, stream=None) -> torch.Tensor:
    band = torch.empty(7 * A.n, dtype=torch.float64, device="cuda")
    _check(lib().airga_mat_to_band(A.h, _ptr(band), _stream(stream)), "mat_to_band")
    return band


# ---------------------------------------------------------------------------
# the path
# ---------------------------------------------------------------------------

def assemble_shifted(M: Mat, K: Mat, alpha: float, beta: float, s: float, stream=None) -> Mat:
    out = C.c_void_p()
    _check(lib().airga_assemble_shifted(M.h, K.h, float(alpha), float(beta), float(s),
                                        _stream(stream), C.byref(out)), "assemble_shifted")
    return Mat(out.value, M.n)


def _colmajor(X: torch.Tensor) -> torch.Tensor:
    """(m, n) contiguous view of an n-vector or a column-major n x m block."""
    if X.dim() == 1:
        return X.reshape(1, -1)
    Xc = X.t()
    if not Xc.is_contiguous():
        raise ValueError("blocks must be column-major (the transpose of a contiguous (m, n) tensor)")
    return Xc


def spmv(A: Mat, X: torch.Tensor, Y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Y = A X for an n-vector or a column-major n x m block."""
    Xc = _colmajor(X)
    if Y is None:
        Yc = torch.empty_like(Xc)
        Y = Yc.reshape(-1) if X.dim() == 1 else Yc.t()
    Yc = _colmajor(Y)
    _check(lib().airga_spmv(A.h, _ptr(Xc, torch.float64), _ptr(Yc, torch.float64), Xc.shape[0],
                            _stream(stream)), "spmv")
    return Y


def spai_build(A: Mat, opts: Options | None = None, stream=None,
               pattern: Mat | None = None) -> Precond:
    """SPAI of A on the pattern of `pattern` (default: A's own pattern)."""
    out = C.c_void_p()
    _check(lib().airga_spai_build(A.h, pattern.h if pattern is not None else None,
                                  C.byref(opts) if opts else None, _stream(stream),
                                  C.byref(out)), "spai_build")
    return Precond(out.value, A.n)


def spai_update(P_prev: Precond, A_prev: Mat, A_next: Mat, opts: Options | None = None,
                stream=None) -> Precond:
    out = C.c_void_p()
    _check(lib().airga_spai_update(P_prev.h, A_prev.h, A_next.h,
                                   C.byref(opts) if opts else None, _stream(stream),
                                   C.byref(out)), "spai_update")
    return Precond(out.value, A_next.n)


def precond_apply(P: Precond, r: torch.Tensor, symmetrize: bool = True,
                  z: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    if z is None:
        z = torch.empty_like(r)
    _check(lib().airga_precond_apply(P.h, _ptr(r, torch.float64), _ptr(z, torch.float64),
                                     1 if symmetrize else 0, _stream(stream)), "precond_apply")
    return z


def precond_factor(P: Precond, k: int, stream=None) -> torch.Tensor:
    band = torch.empty(7 * P.n, dtype=torch.float64, device="cuda")
    _check(lib().airga_precond_factor(P.h, int(k), _ptr(band), _stream(stream)),
           "precond_factor")
    return band


def precond_is_banded(P: Precond) -> bool:
    return bool(lib().airga_precond_is_banded(P.h))


def precond_factor_csr(P: Precond, k: int, stream=None):
    """Factor k as (rowptr, col, val) device tensors (rows sorted)."""
    nnz = int(lib().airga_precond_factor_nnz(P.h, int(k)))
    rp = torch.empty(P.n + 1, dtype=torch.int64, device="cuda")
    ci = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
    va = torch.empty(max(nnz, 1), dtype=torch.float64, device="cuda")
    _check(lib().airga_precond_factor_csr(P.h, int(k), _ptr(rp), _ptr(ci), _ptr(va),
                                          _stream(stream)), "precond_factor_csr")
    return rp, ci[:nnz], va[:nnz]


def precond_from_csr(n: int, factors, stream=None) -> Precond:
    """Chain handle from [(rowptr, col, val), ...] device tensors, factor 0 first."""
    factors = list(factors)
    k = len(factors)
    for rp, ci, va in factors:
        _ptr(rp, torch.int64), _ptr(ci, torch.int32), _ptr(va, torch.float64)
    nnz = (C.c_int64 * k)(*[int(ci.numel()) for _, ci, _ in factors])
    rps = (C.c_void_p * k)(*[rp.data_ptr() for rp, _, _ in factors])
    cis = (C.c_void_p * k)(*[ci.data_ptr() for _, ci, _ in factors])
    vas = (C.c_void_p * k)(*[va.data_ptr() for _, _, va in factors])
    out = C.c_void_p()
    _check(lib().airga_precond_from_csr(int(n), k, nnz, rps, cis, vas, _stream(stream),
                                        C.byref(out)), "precond_from_csr")
    return Precond(out.value, n)


def precond_from_bands(bands, stream=None) -> Precond:
    bands = list(bands)
    n = bands[0].numel() // 7
    arr = (C.c_void_p * len(bands))(*[b.data_ptr() for b in bands])
    for b in bands:
        _ptr(b, torch.float64)
    out = C.c_void_p()
    _check(lib().airga_precond_from_bands(n, len(bands), arr, _stream(stream), C.byref(out)),
           "precond_from_bands")
    return Precond(out.value, n)


def precond_status(P: Precond, stream=None):
    """(steps int32[n], colres float64[n], status) of the newest factor."""
    steps = torch.empty(P.n, dtype=torch.int32, device="cuda")
    colres = torch.empty(P.n, dtype=torch.float64, device="cuda")
    st = C.c_int(0)
    _check(lib().airga_precond_status(P.h, _ptr(steps), _ptr(colres), C.byref(st),
                                      _stream(stream)), "precond_status")
    return steps, colres, st.value


def precond_status_code(P: Precond, stream=None) -> int:
    """Status of the newest factor alone (synchronises the stream)."""
    st = C.c_int(0)
    _check(lib().airga_precond_status(P.h, None, None, C.byref(st), _stream(stream)),
           "precond_status")
    return st.value


def pcg_solve(A: Mat, P: Precond | None, F: torch.Tensor, opts: Options | None = None,
              X: torch.Tensor | None = None, want_hist: bool = False, stream=None):
    """Solve A X = F (F: n or n x m column-major, i.e. a contiguous (m, n)
    tensor transposed, or a contiguous n-vector).  Returns a dict with X,
    iters, status, true_relres (device tensors) and res_hist if asked."""
    if F.dim() == 1:
        Fc = F.reshape(1, -1)
    else:
        Fc = F.t().contiguous() if not F.t().is_contiguous() else F.t()
    m = Fc.shape[0]
    o = opts if opts is not None else options()
    if X is None:
        Xc = torch.zeros_like(Fc)
    else:
        Xc = X.reshape(1, -1) if X.dim() == 1 else X.t()
        if not Xc.is_contiguous():
            raise ValueError("X must be column-major (a transposed contiguous (m, n) tensor)")
    iters = torch.zeros(m, dtype=torch.int32, device="cuda")
    status = torch.zeros(m, dtype=torch.int32, device="cuda")
    relres = torch.zeros(m, dtype=torch.float64, device="cuda")
    hist = torch.full((m, o.maxit + 1), float("nan"), dtype=torch.float64, device="cuda") \
        if want_hist else None
    _check(lib().airga_pcg_solve(A.h, P.h if P is not None else None, _ptr(Fc, torch.float64), m,
                                 C.byref(o), _ptr(Xc, torch.float64), _ptr(hist), _ptr(iters),
                                 _ptr(status), _ptr(relres), _stream(stream)), "pcg_solve")
    out = dict(X=Xc.reshape(-1) if F.dim() == 1 else Xc.t(), iters=iters, status=status,
               true_relres=relres)
    if want_hist:
        out["res_hist"] = hist
    return out


def pcg_solve_mv(A: Mat, P: Precond | None, M: Mat, V: torch.Tensor, rhs_scale: float = 1.0,
                 opts: Options | None = None, want_hist: bool = False, stream=None):
    """Solve A X = rhs_scale M V (V an n-vector or column-major n x m block)
    with M V formed inside the solve (AIRGA inner-loop right-hand sides)."""
    Vc = _colmajor(V) if V.dim() == 2 and V.t().is_contiguous() else \
        (V.reshape(1, -1) if V.dim() == 1 else V.t().contiguous())
    m = Vc.shape[0]
    o = opts if opts is not None else options()
    Xc = torch.zeros_like(Vc)
    iters = torch.zeros(m, dtype=torch.int32, device="cuda")
    status = torch.zeros(m, dtype=torch.int32, device="cuda")
    relres = torch.zeros(m, dtype=torch.float64, device="cuda")
    hist = torch.full((m, o.maxit + 1), float("nan"), dtype=torch.float64, device="cuda") \
        if want_hist else None
    _check(lib().airga_pcg_solve_mv(A.h, P.h if P is not None else None, M.h,
                                    _ptr(Vc, torch.float64), float(rhs_scale), m, C.byref(o),
                                    _ptr(Xc, torch.float64), _ptr(hist), _ptr(iters),
                                    _ptr(status), _ptr(relres), _stream(stream)), "pcg_solve_mv")
    out = dict(X=Xc.reshape(-1) if V.dim() == 1 else Xc.t(), iters=iters, status=status,
               true_relres=relres)
    if want_hist:
        out["res_hist"] = hist
    return out


def pcg_solve_mixed(A: Mat, P: Precond | None, F: torch.Tensor, opts: Options | None = None,
                    stream=None):
    """FP32-inner / FP64-refinement solve of A X = F (F an n-vector or a
    column-major n x m block).  Returns X, outer_iters, inner_iters, status,
    true_relres (device tensors)."""
    Fc = _colmajor(F) if F.dim() == 2 and F.t().is_contiguous() else \
        (F.reshape(1, -1) if F.dim() == 1 else F.t().contiguous())
    m = Fc.shape[0]
    o = opts if opts is not None else options()
    Xc = torch.zeros_like(Fc)
    outer = torch.zeros(m, dtype=torch.int32, device="cuda")
    inner = torch.zeros(m, dtype=torch.int32, device="cuda")
    status = torch.zeros(m, dtype=torch.int32, device="cuda")
    relres = torch.zeros(m, dtype=torch.float64, device="cuda")
    _check(lib().airga_pcg_solve_mixed(A.h, P.h if P is not None else None,
                                       _ptr(Fc, torch.float64), m, C.byref(o),
                                       _ptr(Xc, torch.float64), _ptr(outer), _ptr(inner),
                                       _ptr(status), _ptr(relres), _stream(stream)),
           "pcg_solve_mixed")
    return dict(X=Xc.reshape(-1) if F.dim() == 1 else Xc.t(), outer_iters=outer,
                inner_iters=inner, status=status, true_relres=relres)


class Batch:
    """A planned set of independent single-RHS solves run by one launch
    (airga_batch_*).  systems: list of (A, P or None, f, x) with f, x device
    n-vectors (x receives the solution)."""

    def __init__(self, systems, opts: Options | None = None, cost=None, rows_per_cta: int = 0,
                 stream=None, group=None):
        k = len(systems)
        self.systems = systems           # keep handles and buffers alive
        self.iters = torch.zeros(k, dtype=torch.int32, device="cuda")
        self.status = torch.zeros(k, dtype=torch.int32, device="cuda")
        self.relres = torch.zeros(k, dtype=torch.float64, device="cuda")
        Ah = (C.c_void_p * k)(*[s[0].h.value for s in systems])
        any_p = any(s[1] is not None for s in systems)
        Ph = (C.c_void_p * k)(*[(s[1].h.value if s[1] is not None else None) for s in systems])
        Fp = (C.c_void_p * k)(*[s[2].data_ptr() for s in systems])
        Xp = (C.c_void_p * k)(*[s[3].data_ptr() for s in systems])
        cst = (C.c_double * k)(*cost) if cost is not None else None
        grp = (C.c_int32 * k)(*[int(g) for g in group]) if group is not None else None
        o = opts if opts is not None else options()
        self.opts = o
        out = C.c_void_p()
        _check(lib().airga_batch_create(k, Ah, Ph if any_p else None, Fp, Xp, cst, grp,
                                        int(rows_per_cta), C.byref(o), _ptr(self.iters),
                                        _ptr(self.status), _ptr(self.relres), _stream(stream),
                                        C.byref(out)), "batch_create")
        self.h = out

    def solve(self, stream=None):
        _check(lib().airga_batch_solve(self.h, _stream(stream)), "batch_solve")

    def info(self):
        g, rt, rm, ms = C.c_int32(), C.c_int32(), C.c_int32(), C.c_double()
        _check(lib().airga_batch_info(self.h, C.byref(g), C.byref(rt), C.byref(rm), C.byref(ms)),
               "batch_info")
        return dict(grid=g.value, rows_target=rt.value, rows_max=rm.value, makespan=ms.value)

    def __del__(self):
        if getattr(self, "h", None) and self.h.value and _lib is not None:
            _lib.airga_batch_free(self.h)
            self.h = C.c_void_p(None)


def true_residual(A: Mat, X: torch.Tensor, F: torch.Tensor, stream=None) -> torch.Tensor:
    Xc = X.reshape(1, -1) if X.dim() == 1 else X.t()
    Fc = F.reshape(1, -1) if F.dim() == 1 else F.t()
    m = Fc.shape[0]
    out = torch.empty(m, dtype=torch.float64, device="cuda")
    _check(lib().airga_true_residual(A.h, _ptr(Xc, torch.float64), _ptr(Fc, torch.float64), m,
                                     _ptr(out), _stream(stream)), "true_residual")
    return out


FAULT_NONE, FAULT_SKIP_ARRIVAL, FAULT_ALLOC, FAULT_LAUNCH = 0, 1, 2, 3
PCG_KERNEL_AUTO, PCG_KERNEL_GENERIC_GLOBAL, PCG_KERNEL_PAIR, PCG_KERNEL_PAIR_SPLIT = 0, 1, 2, 3
PCG_KERNEL_PAIR_HALF = 4


def debug_force_pcg_kernel(kind: int):
    """Test hook: prefer one CG kernel variant (0 = automatic)."""
    _check(lib().airga_debug_force_pcg_kernel(int(kind)), "debug_force_pcg_kernel")


def debug_set_fault(fault: int):
    _check(lib().airga_debug_set_fault(int(fault)), "debug_set_fault")


def probe_fp64_rate(iters: int = 1 << 16, stream=None):
    """(FP64 FMAs per SM clock, TFLOP/s, ms) of the device (measurement aid)."""
    f, t, ms = C.c_double(), C.c_double(), C.c_double()
    _check(lib().airga_probe_fp64_rate(int(iters), C.byref(f), C.byref(t), C.byref(ms),
                                       _stream(stream)), "probe_fp64_rate")
    return f.value, t.value, ms.value


def probe_read_bw(nbytes: int, passes: int = 20, stream=None):
    """(GB/s, ms) of streaming reads over a device buffer of `nbytes`
    (below the L2 size: L2 read bandwidth; measurement aid)."""
    g, ms = C.c_double(), C.c_double()
    _check(lib().airga_probe_read_bw(int(nbytes), int(passes), C.byref(g), C.byref(ms),
                                     _stream(stream)), "probe_read_bw")
    return g.value, ms.value


def debug_record_placement(buf=None):
    """Make the next CG calls write each CTA's SM index into `buf` (an int32
    device tensor with at least one entry per SM); None turns it off."""
    _check(lib().airga_debug_record_placement(_ptr(buf, torch.int32) if buf is not None else None),
           "debug_record_placement")


def trace_enable(capacity: int = 4096):
    """Turn call tracing on, keeping at most `capacity` unread records (0
    turns it off and discards them)."""
    _check(lib().airga_trace_enable(int(capacity)), "trace_enable")


def trace_read(max_records: int = 4096):
    """The oldest unread trace records (waits for their end events):
    (list of dicts {name, ms, stream}, calls dropped for lack of capacity
    since the previous read)."""
    buf = (TraceRecord * max(1, int(max_records)))()
    n, dropped = C.c_int32(), C.c_int64()
    _check(lib().airga_trace_read(buf, int(max_records), C.byref(n), C.byref(dropped)), "trace_read")
    return ([dict(name=buf[k].name.decode(), ms=buf[k].ms, stream=buf[k].stream or 0)
             for k in range(n.value)], dropped.value)


def stream_hold(microseconds: int, stream=None):
    """Queue a bounded sleep of `microseconds` on `stream` (see sm_share)."""
    _check(lib().airga_stream_hold(int(microseconds), _stream(stream)), "stream_hold")


def debug_pool_used() -> int:
    """Bytes of the library's device pool in use (synchronise first)."""
    v = C.c_int64()
    _check(lib().airga_debug_pool_used(C.byref(v)), "debug_pool_used")
    return v.value


def debug_checked():
    """Bounds-check record of a checked build since the last call:
    (violations, site, index); raises AirgaError (E_UNSUPPORTED) on a normal
    build."""
    v, site, idx = C.c_int64(), C.c_int32(), C.c_int64()
    _check(lib().airga_debug_checked(C.byref(v), C.byref(site), C.byref(idx)), "debug_checked")
    return v.value, site.value, idx.value


def debug_check_selftest(index, bound, site, stream=None):
    """Run the kernels' bounds check once on (index, [0, bound)) in a checked
    build; no memory is accessed at `index`."""
    _check(lib().airga_debug_check_selftest(int(index), int(bound), int(site), _stream(stream)),
           "debug_check_selftest")


def trim():
    _check(lib().airga_trim(), "trim")


# ---------------------------------------------------------------------------
# convenience: beam inputs to device handles
# ---------------------------------------------------------------------------

def beam_mats(beam, stream=None):
    """(M, K) device handles from a workloads.BeamCSR (CSR uploaded, then
    converted to band storage by the library)."""
    rp = torch.from_numpy(beam.rowptr).cuda()
    ci = torch.from_numpy(beam.col).cuda()
    mv = torch.from_numpy(beam.m_val).cuda()
    kv = torch.from_numpy(beam.k_val).cuda()
    M = mat_from_csr(beam.n, rp, ci, mv, stream)
    K = mat_from_csr(beam.n, rp, ci, kv, stream)
    return M, K


# ---------------------------------------------------------------------------
# learned SPAI-column predictor
# ---------------------------------------------------------------------------

def mlp_train_options(**kw) -> MlpTrainOptions:
    o = MlpTrainOptions()
    lib().airga_mlp_train_options_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Mlp:
    """Owning wrapper of an airga_mlp handle (the learned SPAI-column
    predictor: parameters, Adam state and step counter on the device)."""

    def __init__(self, seed: int = 0, stream=None):
        out = C.c_void_p()
        _check(lib().airga_mlp_create(C.c_uint64(int(seed)), _stream(stream), C.byref(out)),
               "mlp_create")
        self.h = out

    def __del__(self):
        if getattr(self, "h", None) and self.h.value and _lib is not None:
            _lib.airga_mlp_free(self.h)
            self.h = C.c_void_p(None)

    def set_params(self, params: torch.Tensor, stream=None):
        _check(lib().airga_mlp_set_params(self.h, _ptr(params, torch.float32), _stream(stream)),
               "mlp_set_params")

    def params(self, stream=None) -> torch.Tensor:
        out = torch.empty(MLP_NPARAM, dtype=torch.float32, device="cuda")
        _check(lib().airga_mlp_get_params(self.h, _ptr(out), _stream(stream)), "mlp_get_params")
        return out

    def status(self, stream=None):
        """(Adam steps done, status code); synchronises the stream."""
        steps, st = C.c_int64(), C.c_int()
        _check(lib().airga_mlp_status(self.h, C.byref(steps), C.byref(st), _stream(stream)),
               "mlp_status")
        return steps.value, st.value

    def forward(self, X: torch.Tensor, stream=None) -> torch.Tensor:
        Y = torch.empty(X.shape[0], MLP_OUT, dtype=torch.float32, device="cuda")
        _check(lib().airga_mlp_forward(self.h, _ptr(X, torch.float32), X.shape[0], _ptr(Y),
                                       _stream(stream)), "mlp_forward")
        return Y

    def grad(self, X, T, mask, idx, stream=None):
        """(mean gradient float32[NPARAM], loss float64[1]) over rows idx."""
        g = torch.empty(MLP_NPARAM, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float64, device="cuda")
        _check(lib().airga_mlp_grad(self.h, _ptr(X, torch.float32), _ptr(T, torch.float32),
                                    _ptr(mask, torch.uint8), X.shape[0], _ptr(idx, torch.int32),
                                    idx.numel(), _ptr(g), _ptr(loss), _stream(stream)),
               "mlp_grad")
        return g, loss

    def train(self, X, T, mask, steps: int, opts: MlpTrainOptions | None = None, idx=None,
              loss_hist: torch.Tensor | None = None, stream=None):
        o = opts if opts is not None else mlp_train_options()
        _check(lib().airga_mlp_train(self.h, _ptr(X, torch.float32), _ptr(T, torch.float32),
                                     _ptr(mask, torch.uint8), X.shape[0], int(steps), C.byref(o),
                                     _ptr(idx, torch.int32), _ptr(loss_hist, torch.float32),
                                     _stream(stream)), "mlp_train")
        return loss_hist

    def spai(self, A: Mat, s: float, alpha: float, beta: float, stream=None) -> Precond:
        out = C.c_void_p()
        _check(lib().airga_mlp_spai(self.h, A.h, float(s), float(alpha), float(beta),
                                    _stream(stream), C.byref(out)), "mlp_spai")
        return Precond(out.value, A.n)


def mlp_features(A: Mat, P: Precond | None, s: float, alpha: float, beta: float,
                 cols: torch.Tensor | None = None, stream=None):
    """(X[count,16] float32, T[count,8] float32 or None, mask[count] uint8 or
    None, flag int32[1]) for the columns `cols` (device int64) or all columns."""
    count = cols.numel() if cols is not None else A.n
    X = torch.empty(count, MLP_IN, dtype=torch.float32, device="cuda")
    T = torch.empty(count, 8, dtype=torch.float32, device="cuda") if P is not None else None
    mask = torch.empty(count, dtype=torch.uint8, device="cuda") if P is not None else None
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    _check(lib().airga_mlp_features(A.h, P.h if P is not None else None, float(s), float(alpha),
                                    float(beta), _ptr(cols, torch.int64), count, _ptr(X), _ptr(T),
                                    _ptr(mask), _ptr(flag), _stream(stream)), "mlp_features")
    return X, T, mask, flag
