"""Python binding of libflz, the C ABI declared in include/flz.h.

Argument marshalling only: every function forwards to the entry point of the
same name in libflz.so, where all of the computation runs (CUDA kernels for
sm_103a plus the host driver). Pointers may be given as Python ints (device or
host addresses), numpy arrays (host) or objects with ``data_ptr()`` such as
torch tensors (device). Failures raise :class:`FlzError` with the library's
status and message. Importing this package does not load the library;
:func:`lib` does, and raises if libflz.so has not been built (there is no
fallback implementation).
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libflz.so")

FLZ_OK = 0
FLZ_ERR_INVALID_ARG = 1
FLZ_ERR_NOT_SYMMETRIC = 2
FLZ_ERR_BAD_CSR = 3
FLZ_ERR_EMPTY_INTERVAL = 4
FLZ_ERR_NOT_CONVERGED = 5
FLZ_ERR_OUT_OF_MEMORY = 6
FLZ_ERR_CUDA = 7
FLZ_ERR_TIMEOUT = 8
FLZ_ERR_CAPACITY = 9
FLZ_ERR_NO_INTERVAL = 10
FLZ_ERR_NOT_SOLVED = 11

FLZ_F64, FLZ_F32, FLZ_BF16 = 0, 1, 2
FLZ_HOST, FLZ_DEVICE = 0, 1
FLZ_PREC_FP64, FLZ_PREC_FP32, FLZ_PREC_BF16, FLZ_PREC_DF64, FLZ_PREC_FX64 = 0, 1, 2, 3, 4
FLZ_REC_FORWARD, FLZ_REC_CLENSHAW = 0, 1
FLZ_ORTHO_AUTO, FLZ_ORTHO_CUDA_CORES, FLZ_ORTHO_TENSOR = 0, 1, 2
FLZ_START_KRYLOV, FLZ_START_SUBSPACE = 0, 1

# Every symbol include/flz.h declares.
EXPORTED = (
    "flz_status_string", "flz_last_error", "flz_params_default",
    "flz_matrix_create_csr", "flz_matrix_destroy", "flz_matrix_info", "flz_matrix_format",
    "flz_filter_apply", "flz_filter_apply_noalloc", "flz_filter_coefficients", "flz_smoothed_step_coefficients", "flz_jackson_factors", "flz_lanczos_sigma_factors", "flz_filter_degree", "flz_damping_coefficients", "flz_spectrum_bounds",
    "flz_band_eigenvalues", "flz_band_eigenvectors", "flz_sym_eig",
    "flz_basis_project", "flz_basis_orthogonalize", "flz_basis_multiply", "flz_measure_alu_peak", "flz_set_wait_limit", "flz_tc_mma_probe", "flz_solver_create", "flz_solver_destroy", "flz_solver_set_interval", "flz_solver_set_start_vectors", "flz_solve", "flz_solve_sliced",
    "flz_get_count", "flz_get_eigenvalues", "flz_get_eigenvectors", "flz_get_residuals", "flz_get_stats", "flz_get_checks",
    "flz_batch_create", "flz_batch_destroy", "flz_batch_solve", "flz_batch_get_count", "flz_batch_get_eigenvalues",
    "flz_batch_get_residuals", "flz_batch_get_eigenvectors", "flz_batch_get_stats",
)


class flz_params(ctypes.Structure):
    _fields_ = [
        ("block_size", ctypes.c_int32), ("degree", ctypes.c_int32), ("degree_eps", ctypes.c_double),
        ("max_degree", ctypes.c_int32), ("tol", ctypes.c_double), ("check_every", ctypes.c_int32),
        ("max_basis", ctypes.c_int32), ("guard", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("bounds_steps", ctypes.c_int32), ("seed", ctypes.c_uint64), ("lmin", ctypes.c_double),
        ("lmax", ctypes.c_double), ("damping", ctypes.c_int32),
        ("recurrence", ctypes.c_int32), ("transition", ctypes.c_double), ("ortho", ctypes.c_int32),
        ("refine", ctypes.c_int32),
        ("start_mode", ctypes.c_int32),
        ("persistent", ctypes.c_int32),
        ("tile_rows", ctypes.c_int32),
    ]


class flz_stats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int64), ("matvecs", ctypes.c_int64), ("count", ctypes.c_int64),
        ("degree", ctypes.c_int32), ("block_size", ctypes.c_int32), ("converged", ctypes.c_int32),
        ("checks", ctypes.c_int32), ("lmin", ctypes.c_double), ("lmax", ctypes.c_double),
        ("c", ctypes.c_double), ("e", ctypes.c_double), ("alpha_mapped", ctypes.c_double),
        ("beta_mapped", ctypes.c_double), ("max_residual", ctypes.c_double), ("ms_bounds", ctypes.c_double),
        ("ms_filter", ctypes.c_double), ("ms_orth", ctypes.c_double), ("ms_check", ctypes.c_double),
        ("ms_total", ctypes.c_double), ("basis_vectors", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64), ("ortho", ctypes.c_int32), ("filter_precision", ctypes.c_int32),
        ("refine_sweeps", ctypes.c_int32), ("refine_degree", ctypes.c_int32), ("ms_refine", ctypes.c_double),
        ("sweep_matvecs", ctypes.c_int64), ("start_used", ctypes.c_int32), ("tile_rows", ctypes.c_int32),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class flz_check(ctypes.Structure):
    _fields_ = [("block_steps", ctypes.c_int64), ("inside", ctypes.c_int64), ("walked", ctypes.c_int32),
                ("outside", ctypes.c_int32), ("all_small", ctypes.c_int32), ("converged", ctypes.c_int32)]


class FlzError(RuntimeError):
    def __init__(self, status: int, name: str, message: str):
        super().__init__(f"{name}: {message}")
        self.status = status


_lib = None
_vp = ctypes.c_void_p
_i32, _i64, _u64, _dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
_pdbl = ctypes.POINTER(ctypes.c_double)


def lib() -> ctypes.CDLL:
    """Loads libflz.so (built by paper_2409_15053_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libflz.so not built at {LIB_PATH}; run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "flz_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "flz_last_error": (ctypes.c_char_p, []),
        "flz_params_default": (ctypes.c_int, [ctypes.POINTER(flz_params)]),
        "flz_matrix_create_csr": (ctypes.c_int, [_i64, _i64, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _i32,
                                                 ctypes.POINTER(_vp)]),
        "flz_matrix_destroy": (ctypes.c_int, [_vp]),
        "flz_matrix_info": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), _pdbl, _pdbl]),
        "flz_matrix_format": (ctypes.c_int, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i64), ctypes.POINTER(_i32)]),
        "flz_filter_apply": (ctypes.c_int, [_vp, _dbl, _dbl, _vp, _i32, _i32, _vp, _vp, _i32, _i32, _vp]),
        "flz_filter_apply_noalloc": (ctypes.c_int, [_i64, _i64, _vp, _vp, _vp, _dbl, _dbl, _vp, _i32, _i32, _vp,
                                                    _vp, _vp]),
        "flz_filter_coefficients": (ctypes.c_int, [_dbl, _dbl, _i32, _vp]),
        "flz_jackson_factors": (ctypes.c_int, [_i32, _vp]),
        "flz_smoothed_step_coefficients": (ctypes.c_int, [_dbl, _dbl, _dbl, _i32, _vp]),
        "flz_lanczos_sigma_factors": (ctypes.c_int, [_i32, _vp]),
        "flz_filter_degree": (ctypes.c_int, [_dbl, _dbl, _dbl, _i32, ctypes.POINTER(_i32)]),
        "flz_damping_coefficients": (ctypes.c_int, [_dbl, _i32, _vp]),
        "flz_spectrum_bounds": (ctypes.c_int, [_vp, _i32, _i32, _u64, _pdbl, _pdbl, _vp]),
        "flz_band_eigenvalues": (ctypes.c_int, [_i32, _i32, _vp, _vp]),
        "flz_band_eigenvectors": (ctypes.c_int, [_i32, _i32, _vp, _vp, _i32, _vp, _vp, _u64]),
        "flz_sym_eig": (ctypes.c_int, [_i32, _vp, _vp, _vp]),
        "flz_basis_project": (ctypes.c_int, [_i64, _i32, _i32, _vp, _vp, _vp, _i32, _vp]),
        "flz_basis_multiply": (ctypes.c_int, [_i64, _i32, _i32, _vp, _vp, _i32, _vp, _i32, _vp]),
        "flz_measure_alu_peak": (ctypes.c_int, [_i32, _pdbl]),
        "flz_set_wait_limit": (ctypes.c_int, [_u64, ctypes.POINTER(_u64)]),
        "flz_basis_orthogonalize": (ctypes.c_int, [_i64, _i32, _i32, _vp, _vp, _vp, _i32, _vp]),
        "flz_tc_mma_probe": (ctypes.c_int, [_vp, _i64, _vp, _i64, _i32, _i32, _i32, _i32, _i32, _i32, _vp]),
        "flz_solver_create": (ctypes.c_int, [_vp, ctypes.POINTER(flz_params), ctypes.POINTER(_vp)]),
        "flz_solver_destroy": (ctypes.c_int, [_vp]),
        "flz_solver_set_interval": (ctypes.c_int, [_vp, _dbl, _dbl]),
        "flz_solver_set_start_vectors": (ctypes.c_int, [_vp, _vp, _i64, _i32, ctypes.c_int]),
        "flz_solve": (ctypes.c_int, [_vp, _vp]),
        "flz_solve_sliced": (ctypes.c_int, [_vp, _i32, _vp]),
        "flz_get_count": (ctypes.c_int, [_vp, ctypes.POINTER(_i64)]),
        "flz_get_eigenvalues": (ctypes.c_int, [_vp, _vp, _i64]),
        "flz_get_eigenvectors": (ctypes.c_int, [_vp, _vp, _i64, _i64, ctypes.c_int]),
        "flz_get_residuals": (ctypes.c_int, [_vp, _vp, _i64]),
        "flz_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(flz_stats)]),
        "flz_get_checks": (ctypes.c_int, [_vp, _vp, _i64, ctypes.POINTER(_i64)]),
        "flz_batch_create": (ctypes.c_int, [_i32, ctypes.POINTER(_vp), _vp, _vp, ctypes.POINTER(flz_params),
                                            ctypes.POINTER(_vp)]),
        "flz_batch_destroy": (ctypes.c_int, [_vp]),
        "flz_batch_solve": (ctypes.c_int, [_vp, _vp]),
        "flz_batch_get_count": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(_i64)]),
        "flz_batch_get_eigenvalues": (ctypes.c_int, [_vp, _i32, _vp, _i64]),
        "flz_batch_get_residuals": (ctypes.c_int, [_vp, _i32, _vp, _i64]),
        "flz_batch_get_eigenvectors": (ctypes.c_int, [_vp, _i32, _vp, _i64, _i64, ctypes.c_int]),
        "flz_batch_get_stats": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(flz_stats)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int, allow=()):
    if status != FLZ_OK and status not in allow:
        L = lib()
        raise FlzError(status, L.flz_status_string(status).decode(), L.flz_last_error().decode())
    return status


def _ptr(x):
    """Address of a numpy array (host), a tensor with data_ptr() (device), or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy arguments must be C-contiguous")
        return int(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)!r}")


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


def flz_status_string(status: int) -> str:
    return lib().flz_status_string(status).decode()


def flz_last_error() -> str:
    return lib().flz_last_error().decode()


def flz_params_default() -> flz_params:
    p = flz_params()
    _check(lib().flz_params_default(ctypes.byref(p)))
    return p


def flz_matrix_create_csr(n, nnz, rowptr, col, val, val_type=FLZ_F64, where=FLZ_HOST, check_symmetry=1):
    h = _vp()
    _check(lib().flz_matrix_create_csr(int(n), int(nnz), _ptr(rowptr), _ptr(col), _ptr(val), int(val_type),
                                       int(where), int(check_symmetry), ctypes.byref(h)))
    return h


def flz_matrix_destroy(A):
    _check(lib().flz_matrix_destroy(A))


def flz_matrix_info(A):
    n, nnz, glo, ghi = _i64(), _i64(), _dbl(), _dbl()
    _check(lib().flz_matrix_info(A, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(glo), ctypes.byref(ghi)))
    return n.value, nnz.value, glo.value, ghi.value


def flz_matrix_format(A):
    """(sell, sell_entries, long_rows) of the filter's storage of A."""
    sell, entries, long_rows = _i32(), _i64(), _i32()
    _check(lib().flz_matrix_format(A, ctypes.byref(sell), ctypes.byref(entries), ctypes.byref(long_rows)))
    return sell.value, entries.value, long_rows.value


def _coefficients(coeffs, degree):
    coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
    if coeffs.ndim != 1 or coeffs.shape[0] < int(degree) + 1:
        raise ValueError(f"need degree + 1 = {int(degree) + 1} coefficients, got {coeffs.size}")
    return coeffs


def flz_filter_apply(A, c, e, coeffs, degree, r, V, W, precision=FLZ_PREC_FP64, stream=None,
                     recurrence=FLZ_REC_FORWARD):
    coeffs = _coefficients(coeffs, degree)
    _check(lib().flz_filter_apply(A, float(c), float(e), _ptr(coeffs), int(degree), int(r), _ptr(V), _ptr(W),
                                  int(precision), int(recurrence), _stream(stream)))


def flz_filter_apply_noalloc(n, nnz, rowptr, col, val, c, e, coeffs, degree, r, V, W, stream=None):
    """FP64 filter from caller-owned device CSR arrays and blocks; allocates no device memory."""
    coeffs = _coefficients(coeffs, degree)
    _check(lib().flz_filter_apply_noalloc(int(n), int(nnz), _ptr(rowptr), _ptr(col), _ptr(val), float(c), float(e),
                                          _ptr(coeffs), int(degree), int(r), _ptr(V), _ptr(W), _stream(stream)))


def flz_filter_coefficients(alpha, beta, degree) -> np.ndarray:
    out = np.empty(int(degree) + 1)
    _check(lib().flz_filter_coefficients(float(alpha), float(beta), int(degree), _ptr(out)))
    return out


def flz_smoothed_step_coefficients(alpha, beta, delta, degree) -> np.ndarray:
    out = np.empty(int(degree) + 1)
    _check(lib().flz_smoothed_step_coefficients(float(alpha), float(beta), float(delta), int(degree), _ptr(out)))
    return out


def flz_jackson_factors(degree) -> np.ndarray:
    out = np.empty(int(degree) + 1)
    _check(lib().flz_jackson_factors(int(degree), _ptr(out)))
    return out


def flz_damping_coefficients(zc, degree) -> np.ndarray:
    out = np.empty(int(degree) + 1)
    _check(lib().flz_damping_coefficients(float(zc), int(degree), _ptr(out)))
    return out


def flz_lanczos_sigma_factors(degree) -> np.ndarray:
    out = np.empty(int(degree) + 1)
    _check(lib().flz_lanczos_sigma_factors(int(degree), _ptr(out)))
    return out


def flz_filter_degree(alpha, beta, eps=0.3123, max_degree=2000) -> int:
    m = _i32()
    _check(lib().flz_filter_degree(float(alpha), float(beta), float(eps), int(max_degree), ctypes.byref(m)))
    return m.value


def flz_spectrum_bounds(A, steps=60, r=3, seed=1, stream=None):
    lo, hi = _dbl(), _dbl()
    _check(lib().flz_spectrum_bounds(A, int(steps), int(r), int(seed), ctypes.byref(lo), ctypes.byref(hi),
                                     _stream(stream)))
    return lo.value, hi.value


def flz_band_eigenvalues(T: np.ndarray, b: int) -> np.ndarray:
    T = np.ascontiguousarray(T, dtype=np.float64)
    K = T.shape[0]
    theta = np.empty(K)
    _check(lib().flz_band_eigenvalues(K, int(b), _ptr(T), _ptr(theta)))
    return theta


def flz_band_eigenvectors(T: np.ndarray, b: int, theta: np.ndarray, idx, seed: int = 1) -> np.ndarray:
    """(K, count) unit eigenvectors for theta[idx]."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    K = T.shape[0]
    Y = np.empty((idx.shape[0], K))  # row t = column t of the column-major result
    _check(lib().flz_band_eigenvectors(K, int(b), _ptr(T), _ptr(theta), int(idx.shape[0]), _ptr(idx), _ptr(Y),
                                       int(seed)))
    return Y.T


def flz_sym_eig(S: np.ndarray):
    """(w, Z): ascending eigenvalues and eigenvectors (columns) of a dense symmetric matrix."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    n = S.shape[0]
    w = np.empty(n)
    Z = np.empty((n, n))
    _check(lib().flz_sym_eig(n, _ptr(S), _ptr(w), _ptr(Z)))
    return w, Z



def flz_basis_project(n, nb, r, Q, W, C, method=FLZ_ORTHO_TENSOR, stream=None):
    """C = Q^T W for a basis of nb device blocks (n x r each, contiguous) and device W, C."""
    _check(lib().flz_basis_project(int(n), int(nb), int(r), _ptr(Q), _ptr(W), _ptr(C), int(method),
                                   _stream(stream)))


def flz_basis_orthogonalize(n, nb, r, Q, W, C, method=FLZ_ORTHO_TENSOR, stream=None):
    """W <- (I - QQ^T)^2 W in place; C = total projection coefficients (device)."""
    _check(lib().flz_basis_orthogonalize(int(n), int(nb), int(r), _ptr(Q), _ptr(W), _ptr(C), int(method),
                                         _stream(stream)))


def flz_basis_multiply(n, nb, r, Q, H, s, X, method=FLZ_ORTHO_TENSOR, stream=None):
    """X = Q H for a basis of nb device blocks, H (nb r x s) and X (n x s) device, row-major."""
    _check(lib().flz_basis_multiply(int(n), int(nb), int(r), _ptr(Q), _ptr(H), int(s), _ptr(X), int(method),
                                    _stream(stream)))


def flz_measure_alu_peak(kind) -> float:
    """Measured FP64 FMA (kind 0) or 32-bit integer multiply-add (kind 1) rate, operations per second."""
    out = ctypes.c_double()
    _check(lib().flz_measure_alu_peak(int(kind), ctypes.byref(out)))
    return out.value


def flz_set_wait_limit(ns) -> int:
    """Sets the device wait limit (ns) of later kernels; returns the previous limit."""
    prev = _u64()
    _check(lib().flz_set_wait_limit(int(ns), ctypes.byref(prev)))
    return prev.value


def flz_tc_mma_probe(a_img, b_img, n, a_mn_major, a_lbo, a_sbo, b_lbo, b_sbo):
    """One tcgen05 MMA of shared-memory images (uint16 arrays); returns D (128 x n, float32)."""
    a_img = np.ascontiguousarray(a_img, dtype=np.uint16)
    b_img = np.ascontiguousarray(b_img, dtype=np.uint16)
    d = np.zeros((128, int(n)), dtype=np.float32)
    _check(lib().flz_tc_mma_probe(_ptr(a_img), a_img.nbytes, _ptr(b_img), b_img.nbytes, int(n), int(a_mn_major),
                                  int(a_lbo), int(a_sbo), int(b_lbo), int(b_sbo), _ptr(d)))
    return d

def flz_solver_create(A, params: flz_params | None = None):
    h = _vp()
    _check(lib().flz_solver_create(A, ctypes.byref(params) if params is not None else None, ctypes.byref(h)))
    return h


def flz_solver_destroy(s):
    _check(lib().flz_solver_destroy(s))


def flz_solver_set_interval(s, alpha, beta):
    _check(lib().flz_solver_set_interval(s, float(alpha), float(beta)))


def flz_solver_set_start_vectors(s, X, ld=None, where=None):
    """Warm start: the next solves start from combinations of the columns of X (n x cols, column-major).

    X may be a host numpy array of shape (n, cols) (any layout; copied column-major) or a device tensor
    holding the columns contiguously (ld = n) with where=FLZ_DEVICE; None clears the start vectors."""
    if X is None:
        _check(lib().flz_solver_set_start_vectors(s, None, 0, 0, FLZ_HOST))
        return
    if isinstance(X, np.ndarray):
        Xc = np.asfortranarray(X, dtype=np.float64)
        n, cols = Xc.shape
        _check(lib().flz_solver_set_start_vectors(s, int(Xc.ctypes.data), int(n), int(cols), FLZ_HOST))
        return
    n, cols = int(X.shape[0]), int(X.shape[1])
    _check(lib().flz_solver_set_start_vectors(s, _ptr(X), int(ld if ld is not None else n), cols,
                                              FLZ_DEVICE if where is None else int(where)))


def flz_solve(s, stream=None) -> int:
    """Returns FLZ_OK or FLZ_ERR_NOT_CONVERGED (partial results readable); raises on other failures."""
    return _check(lib().flz_solve(s, _stream(stream)), allow=(FLZ_ERR_NOT_CONVERGED,))


def flz_solve_sliced(s, nslices, stream=None) -> int:
    """Spectrum slicing over nslices equal-width sub-intervals; results merged into s."""
    return _check(lib().flz_solve_sliced(s, int(nslices), _stream(stream)), allow=(FLZ_ERR_NOT_CONVERGED,))


def flz_get_count(s) -> int:
    c = _i64()
    _check(lib().flz_get_count(s, ctypes.byref(c)))
    return c.value


def flz_get_eigenvalues(s, out=None) -> np.ndarray:
    cnt = flz_get_count(s)
    out = np.empty(max(cnt, 1)) if out is None else out
    _check(lib().flz_get_eigenvalues(s, _ptr(out), int(out.shape[0])))
    return out[:cnt]


def flz_get_residuals(s, out=None) -> np.ndarray:
    cnt = flz_get_count(s)
    out = np.empty(max(cnt, 1)) if out is None else out
    _check(lib().flz_get_residuals(s, _ptr(out), int(out.shape[0])))
    return out[:cnt]


def flz_get_eigenvectors(s, out, ld, cap_cols, where=FLZ_HOST):
    """Writes the n x count column-major eigenvectors (leading dimension ld) into `out`."""
    _check(lib().flz_get_eigenvectors(s, _ptr(out), int(ld), int(cap_cols), int(where)))
    return out


def get_eigenvectors_host(s, n: int) -> np.ndarray:
    """(n, count) float64 eigenvectors copied to the host (column j matches eigenvalue j)."""
    cnt = flz_get_count(s)
    buf = np.empty((max(cnt, 1), n))  # row t of buf = column t of the column-major result
    _check(lib().flz_get_eigenvectors(s, _ptr(buf), int(n), int(max(cnt, 1)), FLZ_HOST))
    return buf[:cnt].T


def flz_get_checks(s) -> list:
    """The convergence checks of the last solve, as dicts (block_steps, inside, walked, outside, ...)."""
    cnt = _i64()
    _check(lib().flz_get_checks(s, None, 0, ctypes.byref(cnt)))
    arr = (flz_check * max(cnt.value, 1))()
    _check(lib().flz_get_checks(s, arr, cnt.value, None))
    return [{name: getattr(arr[i], name) for name, _ in flz_check._fields_} for i in range(cnt.value)]


def flz_get_stats(s) -> dict:
    st = flz_stats()
    _check(lib().flz_get_stats(s, ctypes.byref(st)))
    return st.as_dict()


def flz_batch_create(mats, alphas, betas, params: flz_params | None = None):
    """Batch of independent problems; `mats` are matrix handles that must outlive the batch."""
    count = len(mats)
    arr = (_vp * count)(*[m.value if isinstance(m, _vp) else m for m in mats])
    a = np.ascontiguousarray(alphas, dtype=np.float64)
    b = np.ascontiguousarray(betas, dtype=np.float64)
    h = _vp()
    _check(lib().flz_batch_create(count, arr, _ptr(a), _ptr(b), ctypes.byref(params) if params is not None else None,
                                  ctypes.byref(h)))
    return h


def flz_batch_destroy(b):
    _check(lib().flz_batch_destroy(b))


def flz_batch_solve(b, stream=None) -> int:
    return _check(lib().flz_batch_solve(b, _stream(stream)), allow=(FLZ_ERR_NOT_CONVERGED,))


def flz_batch_get_count(b, index) -> int:
    c = _i64()
    _check(lib().flz_batch_get_count(b, int(index), ctypes.byref(c)))
    return c.value


def flz_batch_get_eigenvalues(b, index) -> np.ndarray:
    cnt = flz_batch_get_count(b, index)
    out = np.empty(max(cnt, 1))
    _check(lib().flz_batch_get_eigenvalues(b, int(index), _ptr(out), int(out.shape[0])))
    return out[:cnt]


def flz_batch_get_residuals(b, index) -> np.ndarray:
    cnt = flz_batch_get_count(b, index)
    out = np.empty(max(cnt, 1))
    _check(lib().flz_batch_get_residuals(b, int(index), _ptr(out), int(out.shape[0])))
    return out[:cnt]


def flz_batch_get_eigenvectors(b, index, out, ld, cap_cols, where=FLZ_HOST):
    _check(lib().flz_batch_get_eigenvectors(b, int(index), _ptr(out), int(ld), int(cap_cols), int(where)))
    return out


def batch_eigenvectors_host(b, index, n: int) -> np.ndarray:
    """(n, count) eigenvectors of problem `index` copied to the host."""
    cnt = flz_batch_get_count(b, index)
    buf = np.empty((max(cnt, 1), n))
    _check(lib().flz_batch_get_eigenvectors(b, int(index), _ptr(buf), int(n), int(max(cnt, 1)), FLZ_HOST))
    return buf[:cnt].T


def flz_batch_get_stats(b, index) -> dict:
    st = flz_stats()
    _check(lib().flz_batch_get_stats(b, int(index), ctypes.byref(st)))
    return st.as_dict()
