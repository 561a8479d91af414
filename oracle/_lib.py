"""ctypes loader of the oracle's C library (test infrastructure only)."""
import ctypes
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None


class OraGrid(ctypes.Structure):
    """Mirror of `ora_grid` in fwi_oracle.c."""
    _fields_ = [
        ("dims", ctypes.c_int), ("nz", ctypes.c_int), ("ny", ctypes.c_int),
        ("nx", ctypes.c_int), ("nbl", ctypes.c_int), ("so", ctypes.c_int),
        ("nt", ctypes.c_int), ("h", ctypes.c_double), ("dt", ctypes.c_double),
        ("vmax_damp", ctypes.c_double), ("refl", ctypes.c_double),
        ("time_order", ctypes.c_int),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i = ctypes.c_int
            L.ora_fd_weights.argtypes = [i, P]
            L.ora_laplacian.argtypes = [P, P, P]
            L.ora_damping.argtypes = [P, P]
            L.ora_ricker.argtypes = [i, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, P]
            L.ora_interp.argtypes = [P, P, P, P]
            L.ora_forward.argtypes = [P, P, i, P, P, i, P, P, P]
            L.ora_step.argtypes = [P, P, P, P, P]
            L.ora_adjoint.argtypes = [P, P, i, P, P, i, P, P, P, P, P, i]
            L.ora_gradient.argtypes = [P, P, i, P, P, i, P, P, P, P, P, i]
            L.ora_problem_create.argtypes = [P, P, i, P, P, i, P]
            L.ora_problem_create.restype = P
            L.ora_problem_destroy.argtypes = [P]
            L.ora_problem_destroy.restype = None
            L.ora_problem_fwd_step.argtypes = [P, i, P, P, P]
            L.ora_problem_adj_step.argtypes = [P, P, i, P, P, P, P, P]
            L.codec_compress.argtypes = [i, i, i, i, P, ctypes.c_double, P, ctypes.c_size_t, P]
            L.codec_compress.restype = ctypes.c_longlong
            L.codec_decompress.argtypes = [i, i, i, i, P, ctypes.c_size_t, P]
            L.codec_bound_words.argtypes = [i, i, i, i]
            L.codec_bound_words.restype = ctypes.c_longlong
            L.codec_compress_rate.argtypes = [i, i, i, i, P, i, P, ctypes.c_size_t, P]
            L.codec_compress_rate.restype = ctypes.c_longlong
            L.codec_rate_words.argtypes = [i, i, i, i, i]
            L.codec_rate_words.restype = ctypes.c_longlong
            for f in ("ora_fd_weights", "ora_laplacian", "ora_damping", "ora_ricker",
                      "ora_interp", "ora_forward", "ora_step", "ora_adjoint", "ora_gradient",
                      "ora_problem_fwd_step", "ora_problem_adj_step",
                      "codec_decompress"):
                getattr(L, f).restype = ctypes.c_int
            _lib = L
    return _lib
