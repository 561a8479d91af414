"""Fixed-accuracy and fixed-rate 4^d block-transform codec (test
infrastructure only).

numpy front end of codec_oracle.c, whose header holds the full
specification.  The paper stores checkpoints with ZFP's fixed-tolerance
mode, an absolute point-wise error bound (Sec. 2.2 "Lossy Compression");
this codec is an independently specified member of that family.
"""
import ctypes

import numpy as np

from ._lib import lib

STATUS = {0: "ok", -1: "EINVAL", -2: "ENOMEM", -3: "OVERFLOW", -4: "CORRUPT"}


def _shape3(x, dims):
    if dims == 3:
        nz, ny, nx = x.shape
    else:
        nz, nx = x.shape
        ny = 1
    return nz, ny, nx


def bound_words(shape, dims):
    nz, ny, nx = (shape if dims == 3 else (shape[0], 1, shape[1]))
    return int(lib().codec_bound_words(dims, nz, ny, nx))


def compress(x, tol):
    """Compress a float32 2D/3D field; returns (stream uint32 array, nonfinite flag)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    dims = x.ndim
    nz, ny, nx = _shape3(x, dims)
    cap = bound_words(x.shape, dims)
    out = np.zeros(cap, dtype=np.uint32)
    flags = ctypes.c_int(0)
    n = lib().codec_compress(dims, nz, ny, nx, x.ctypes.data_as(ctypes.c_void_p), float(tol),
                             out.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(flags))
    if n < 0:
        raise ValueError("codec_compress: %s" % STATUS.get(int(n), n))
    return out[:n].copy(), bool(flags.value)


def rate_words(shape, dims, rate):
    """Words of a fixed-rate stream: 16 + nblocks * ceil(rate * 4^dims / 32)."""
    nz, ny, nx = (shape if dims == 3 else (shape[0], 1, shape[1]))
    return int(lib().codec_rate_words(dims, nz, ny, nx, int(rate)))


def compress_rate(x, rate):
    """Fixed-rate compression (rate bits per value, 1..32); returns
    (stream uint32 array, nonfinite flag)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    dims = x.ndim
    nz, ny, nx = _shape3(x, dims)
    cap = rate_words(x.shape, dims, rate)
    if cap < 0:
        raise ValueError("codec_rate_words: %s" % STATUS.get(int(cap), cap))
    out = np.zeros(cap, dtype=np.uint32)
    flags = ctypes.c_int(0)
    n = lib().codec_compress_rate(dims, nz, ny, nx, x.ctypes.data_as(ctypes.c_void_p), int(rate),
                                  out.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(flags))
    if n < 0:
        raise ValueError("codec_compress_rate: %s" % STATUS.get(int(n), n))
    return out[:n].copy(), bool(flags.value)


def decompress(stream, shape):
    stream = np.ascontiguousarray(np.asarray(stream, dtype=np.uint32))
    dims = len(shape)
    out = np.zeros(shape, dtype=np.float32)
    nz, ny, nx = _shape3(out, dims)
    st = lib().codec_decompress(dims, nz, ny, nx, stream.ctypes.data_as(ctypes.c_void_p),
                                stream.size, out.ctypes.data_as(ctypes.c_void_p))
    if st != 0:
        raise ValueError("codec_decompress: %s" % STATUS.get(int(st), st))
    return out


def block_stats(stream, shape):
    """[nblocks][5]: bits, mode (0 zero / 1 coded / 2 raw), ptop, pbot, Emax."""
    stream = np.ascontiguousarray(np.asarray(stream, dtype=np.uint32))
    dims = len(shape)
    nb = int(stream[5])
    out = np.zeros((nb, 5), dtype=np.int32)
    nz, ny, nx = (shape if dims == 3 else (shape[0], 1, shape[1]))
    L = lib()
    L.codec_block_stats.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p, ctypes.c_size_t,
                                                         ctypes.c_void_p]
    st = L.codec_block_stats(dims, nz, ny, nx, stream.ctypes.data_as(ctypes.c_void_p),
                             stream.size, out.ctypes.data_as(ctypes.c_void_p))
    if st != 0:
        raise ValueError("codec_block_stats: %s" % STATUS.get(int(st), st))
    return out


def ratio(stream, shape):
    """Compression ratio F = raw float bytes / stream bytes."""
    return float(np.prod(shape)) * 4.0 / (4.0 * len(stream))
