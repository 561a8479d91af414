"""ctypes loader of libckfwi.so (the C-ABI declared in include/ckfwi.h).

The library is built in-tree by paper_1810_05268_gb300/build.py.  There is
no fallback: if the shared library is missing or fails to load, every call
raises.
"""
import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libckfwi.so")

_lock = threading.Lock()
_lib = None


class Grid(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int), ("n", ctypes.c_int * 3), ("nbl", ctypes.c_int),
                ("h", ctypes.c_double), ("space_order", ctypes.c_int), ("dt", ctypes.c_double),
                ("nt", ctypes.c_int), ("vmax_damp", ctypes.c_double), ("time_order", ctypes.c_int)]


class Shot(ctypes.Structure):
    _fields_ = [("src", ctypes.c_double * 3), ("f0", ctypes.c_double), ("t0", ctypes.c_double),
                ("amp", ctypes.c_double), ("wavelet", ctypes.c_void_p), ("nrec", ctypes.c_int),
                ("rec", ctypes.c_void_p)]


class GradOpts(ctypes.Structure):
    _fields_ = [("ckpt_slots", ctypes.c_int), ("store_mode", ctypes.c_int), ("tol", ctypes.c_double),
                ("pool_bytes", ctypes.c_size_t), ("grad_kind", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("profile", ctypes.c_int), ("grad_scale", ctypes.c_double), ("grad_f32", ctypes.c_int),
                ("host_slots", ctypes.c_int), ("rate", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("fwd_steps", ctypes.c_longlong), ("adj_steps", ctypes.c_longlong), ("p", ctypes.c_longlong),
                ("takeshots", ctypes.c_longlong), ("restores", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong), ("pool_bytes_peak", ctypes.c_double),
                ("ratio_min", ctypes.c_double), ("ratio_mean", ctypes.c_double),
                ("u_absmax", ctypes.c_double), ("fwd_ms", ctypes.c_double), ("adj_ms", ctypes.c_double),
                ("comp_ms", ctypes.c_double), ("decomp_ms", ctypes.c_double), ("other_ms", ctypes.c_double),
                ("fwd_launches", ctypes.c_longlong), ("adj_launches", ctypes.c_longlong),
                ("comp_calls", ctypes.c_longlong), ("decomp_calls", ctypes.c_longlong),
                ("fwd_ver", ctypes.c_int), ("fwd_bx", ctypes.c_int), ("fwd_by", ctypes.c_int),
                ("fwd_vec", ctypes.c_int), ("fwd_zlen", ctypes.c_int),
                ("adj_ver", ctypes.c_int), ("adj_bx", ctypes.c_int), ("adj_by", ctypes.c_int),
                ("adj_vec", ctypes.c_int), ("adj_zlen", ctypes.c_int),
                ("fwd_pf", ctypes.c_int), ("adj_pf", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ["ckfwi_create_model", "ckfwi_set_model", "ckfwi_forward_shot", "ckfwi_misfit", "ckfwi_adjoint_gradient",
           "ckfwi_batch_gradient", "ckfwi_batch_gradient_models", "ckfwi_free", "ckfwi_error_string", "ckfwi_revolve_schedule",
           "ckfwi_multistage_schedule", "ckfwi_codec_bound_words", "ckfwi_codec_compress", "ckfwi_codec_decompress",
           "ckfwi_codec_compress_noalloc", "ckfwi_codec_rate_words", "ckfwi_codec_compress_rate", "ckfwi_stream_words"]


def lib():
    """Load (once) and return the library; raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libckfwi.so is not built (%s); run paper_1810_05268_gb300/build.py "
                               "or __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P, I, LL, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
        L.ckfwi_create_model.argtypes = [P, P]
        L.ckfwi_set_model.argtypes = [P, P, I, I, P]
        L.ckfwi_forward_shot.argtypes = [P, P, P, I, P]
        L.ckfwi_misfit.argtypes = [P, P, P, I, P, P, P]
        L.ckfwi_adjoint_gradient.argtypes = [P, P, P, I, P, P, P, P, P]
        L.ckfwi_batch_gradient.argtypes = [P, P, I, P, I, P, P, P, P, P]
        L.ckfwi_batch_gradient_models.argtypes = [P, P, I, P, I, P, P, P, P, P, P, P]
        L.ckfwi_free.argtypes = [P]
        L.ckfwi_free.restype = None
        L.ckfwi_error_string.argtypes = [I]
        L.ckfwi_error_string.restype = ctypes.c_char_p
        L.ckfwi_revolve_schedule.argtypes = [I, I, P, LL, P, P]
        L.ckfwi_multistage_schedule.argtypes = [I, I, I, P, LL, P, P]
        L.ckfwi_codec_bound_words.argtypes = [I, I, I, I]
        L.ckfwi_codec_bound_words.restype = LL
        L.ckfwi_codec_compress.argtypes = [P, I, I, I, I, D, P, LL, P, P, P]
        L.ckfwi_codec_decompress.argtypes = [P, LL, I, I, I, I, P, P]
        L.ckfwi_codec_compress_noalloc.argtypes = [P, I, I, I, I, D, P, LL, P, P, P]
        L.ckfwi_stream_words.argtypes = [P, P, LL, P]
        L.ckfwi_codec_rate_words.argtypes = [I, I, I, I, I]
        L.ckfwi_codec_rate_words.restype = LL
        L.ckfwi_codec_compress_rate.argtypes = [P, I, I, I, I, I, P, LL, P, P, P]
        for name in ("ckfwi_create_model", "ckfwi_set_model", "ckfwi_forward_shot", "ckfwi_misfit",
                     "ckfwi_adjoint_gradient",
                     "ckfwi_batch_gradient", "ckfwi_batch_gradient_models", "ckfwi_revolve_schedule", "ckfwi_multistage_schedule",
                     "ckfwi_codec_compress", "ckfwi_codec_decompress", "ckfwi_codec_compress_noalloc"):
            getattr(L, name).restype = I
        _lib = L
        return _lib


def loaded_path():
    return LIB_PATH if _lib is not None else None
