"""Python binding of the ckfwi C-ABI (include/ckfwi.h): same names,
argument marshalling only.  Every computation runs in libckfwi.so.

Buffers may be torch CUDA tensors (passed as device pointers, work queued on
torch's current stream) or numpy arrays (host memory; the library copies
through its own device buffers).
"""
import ctypes
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from ._lib import GradOpts, Grid, Shot, Stats, lib

OK, EINVAL, ENOMEM, POOL_OVERFLOW, NONFINITE, CORRUPT, TIMEOUT, ECUDA = 0, -1, -2, -3, -4, -5, -6, -7
HOST, DEVICE = 0, 1
STORE_FP32, STORE_BF16, STORE_FP16, STORE_CODEC, STORE_CODEC_RATE = 0, 1, 2, 3, 4
VELOCITY, SLOWNESS2 = 0, 1
STORE_NAMES = {"fp32": STORE_FP32, "bf16": STORE_BF16, "fp16": STORE_FP16, "codec": STORE_CODEC,
               "rate": STORE_CODEC_RATE}


class CkfwiError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (%d)" % (where, error_string(status), status))


def error_string(status):
    return lib().ckfwi_error_string(int(status)).decode()


def _check(st, where):
    if st != OK:
        raise CkfwiError(st, where)


def _is_torch_cuda(x):
    try:
        import torch
    except ImportError:
        return False
    return isinstance(x, torch.Tensor) and x.is_cuda


def _stream(stream=None):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


def _buf(x, dtype):
    """(pointer, mem) of a torch CUDA tensor or a numpy array of `dtype`."""
    if _is_torch_cuda(x):
        import torch
        want = {np.float32: torch.float32, np.float64: torch.float64}[np.dtype(dtype).type]
        if x.dtype != want or not x.is_contiguous():
            raise ValueError("device buffers must be contiguous %s" % np.dtype(dtype).name)
        return ctypes.c_void_p(x.data_ptr()), DEVICE
    a = np.asarray(x)
    if a.dtype != dtype or not a.flags.c_contiguous:
        raise ValueError("host buffers must be contiguous %s" % np.dtype(dtype).name)
    return ctypes.c_void_p(a.ctypes.data), HOST


def _numel(x):
    return int(x.numel()) if _is_torch_cuda(x) else int(np.asarray(x).size)


def _need(x, n, what):
    """The library reads or writes n values of x: refuse a smaller buffer
    here, before a kernel would run past its end."""
    have = _numel(x)
    if have < n:
        raise ValueError("%s holds %d values, the call needs %d" % (what, have, n))


@dataclass
class GridSpec:
    dims: int
    shape: tuple            # total grid (nz, ny, nx) or (nz, nx)
    nbl: int
    h: float                # [m]
    space_order: int
    dt: float               # [ms]
    nt: int
    vmax_damp: float        # [km/s]
    time_order: int = 2     # 2: OT2 kernel, 4: OT4 kernel (Sec. 6)

    def c(self):
        g = Grid()
        g.dims = self.dims
        n = tuple(self.shape) if self.dims == 3 else (self.shape[0], 1, self.shape[1])
        for i in range(3):
            g.n[i] = int(n[i])
        g.nbl, g.h, g.space_order = int(self.nbl), float(self.h), int(self.space_order)
        g.dt, g.nt, g.vmax_damp = float(self.dt), int(self.nt), float(self.vmax_damp)
        g.time_order = int(self.time_order)
        return g

    @property
    def npts(self):
        return int(np.prod(self.shape))


@dataclass
class ShotSpec:
    src: tuple                      # (z, y, x) [m] from the first interior point
    rec: np.ndarray                 # [nrec][3] (z, y, x) [m]
    f0: float = 0.010               # [kHz]
    t0: float = 0.0                 # [ms], <= 0: 1.5/f0
    amp: float = 1.0
    wavelet: Optional[np.ndarray] = None   # [nt] float32 overriding the Ricker
    _keep: list = field(default_factory=list, repr=False)

    def c(self, nt=None):
        """The C struct; with nt, a wavelet shorter than nt samples is refused."""
        s = Shot()
        for i in range(3):
            s.src[i] = float(self.src[i])
        s.f0, s.t0, s.amp = float(self.f0), float(self.t0), float(self.amp)
        rec = np.ascontiguousarray(np.asarray(self.rec, dtype=np.float64).reshape(-1, 3))
        s.nrec = rec.shape[0]
        s.rec = rec.ctypes.data
        self._keep = [rec]
        if self.wavelet is not None:
            w = np.ascontiguousarray(np.asarray(self.wavelet, dtype=np.float32))
            if nt is not None and w.size < nt:
                raise ValueError("the wavelet has %d samples, the grid %d time steps" % (w.size, nt))
            s.wavelet = w.ctypes.data
            self._keep.append(w)
        else:
            s.wavelet = None
        return s

    @property
    def nrec(self):
        return int(np.asarray(self.rec).reshape(-1, 3).shape[0])


def create_model(grid: GridSpec):
    h = ctypes.c_void_p()
    g = grid.c()
    _check(lib().ckfwi_create_model(ctypes.byref(g), ctypes.byref(h)), "ckfwi_create_model")
    return h


def set_model(model, data, kind=VELOCITY, stream=None):
    p, mem = _buf(data, np.float32)
    _check(lib().ckfwi_set_model(model, p, int(kind), mem, _stream(stream)), "ckfwi_set_model")


def forward_shot(model, grid: GridSpec, shot: ShotSpec, d_sim=None, device=None, stream=None):
    """Simulated data [nt+1][nrec] (float32)."""
    if d_sim is None:
        if device is None:
            device = _default_device()
        d_sim = _alloc((grid.nt + 1, shot.nrec), np.float32, device)
    p, mem = _buf(d_sim, np.float32)
    _need(d_sim, (grid.nt + 1) * shot.nrec, "d_sim")
    s = shot.c(grid.nt)
    _check(lib().ckfwi_forward_shot(model, ctypes.byref(s), p, mem, _stream(stream)), "ckfwi_forward_shot")
    return d_sim


def _default_device():
    try:
        import torch
        return "cuda" if torch.cuda.is_available() else None
    except ImportError:
        return None


def _alloc(shape, dtype, device):
    if device is not None:
        import torch
        tdt = {np.float32: torch.float32, np.float64: torch.float64}[dtype]
        return torch.empty(shape, dtype=tdt, device=device)
    return np.empty(shape, dtype=dtype)


def _opts(ckpt_slots, store_mode, tol, pool_bytes, grad_kind, use_graph, profile=False, grad_scale=1.0,
          grad_f32=False, host_slots=0, rate=0):
    o = GradOpts()
    o.ckpt_slots = int(ckpt_slots)
    if isinstance(store_mode, str):
        if store_mode not in STORE_NAMES:
            raise ValueError("unknown store_mode %r (one of %s)" % (store_mode, ", ".join(STORE_NAMES)))
        o.store_mode = STORE_NAMES[store_mode]
    else:
        o.store_mode = int(store_mode)
    o.tol = float(tol)
    o.pool_bytes = int(pool_bytes)
    o.grad_kind = int(grad_kind)
    o.use_graph = int(bool(use_graph))
    o.profile = int(bool(profile))
    o.grad_scale = float(grad_scale)
    o.grad_f32 = int(bool(grad_f32))
    o.host_slots = int(host_slots)
    o.rate = int(rate)
    return o


def misfit(model, grid: GridSpec, shot: ShotSpec, d_obs, d_sim=None, stream=None):
    """phi = 1/2 sum_{n>=1} ||d_sim^n - d_obs^n||^2 (FP64) by forward modelling only."""
    pd, mem = _buf(d_obs, np.float32)
    _need(d_obs, (grid.nt + 1) * shot.nrec, "d_obs")
    ps = None
    if d_sim is not None:
        ps, ms = _buf(d_sim, np.float32)
        if ms != mem:
            raise ValueError("d_obs and d_sim must both be host or both be device buffers")
        _need(d_sim, (grid.nt + 1) * shot.nrec, "d_sim")
    s = shot.c(grid.nt)
    phi = ctypes.c_double(0.0)
    _check(lib().ckfwi_misfit(model, ctypes.byref(s), pd, mem, ctypes.byref(phi), ps, _stream(stream)),
           "ckfwi_misfit")
    return phi.value


def adjoint_gradient(model, grid: GridSpec, shot: ShotSpec, d_obs, ckpt_slots, store_mode=STORE_FP32,
                     tol=0.0, pool_bytes=0, grad_kind=SLOWNESS2, use_graph=False, grad=None, stream=None,
                     profile=False, grad_scale=1.0, host_slots=0, rate=0):
    """(misfit, gradient on the total grid, stats dict)."""
    pd, mem = _buf(d_obs, np.float32)
    if grad is None:
        grad = _alloc(tuple(grid.shape), np.float32, "cuda" if mem == DEVICE else None)
    pg, memg = _buf(grad, np.float32)
    if memg != mem:
        raise ValueError("d_obs and grad must both be host or both be device buffers")
    _need(d_obs, (grid.nt + 1) * shot.nrec, "d_obs")
    _need(grad, grid.npts, "grad")
    s = shot.c(grid.nt)
    o = _opts(ckpt_slots, store_mode, tol, pool_bytes, grad_kind, use_graph, profile, grad_scale,
              host_slots=host_slots, rate=rate)
    phi = ctypes.c_double(0.0)
    st = Stats()
    _check(lib().ckfwi_adjoint_gradient(model, ctypes.byref(s), pd, mem, ctypes.byref(o), ctypes.byref(phi), pg,
                                        ctypes.byref(st), _stream(stream)), "ckfwi_adjoint_gradient")
    return phi.value, grad, st.as_dict()


def _d_obs_ptrs(d_obs_list):
    n = len(d_obs_list)
    ptrs = (ctypes.c_void_p * n)()
    mem = None
    for i, d in enumerate(d_obs_list):
        p, m = _buf(d, np.float32)
        ptrs[i] = p
        if mem is not None and m != mem:
            raise ValueError("mixed host / device d_obs")
        mem = m
    return ptrs, mem


def _shot_array(shots, nt=None):
    carr = (Shot * len(shots))()
    keep = []
    for i, sh in enumerate(shots):
        carr[i] = sh.c(nt)
        keep.append(sh._keep)
    return carr, keep


def batch_gradient(model, grid: GridSpec, shots, d_obs_list, ckpt_slots, store_mode=STORE_FP32, tol=0.0,
                   pool_bytes=0, grad_kind=SLOWNESS2, use_graph=False, grad_sum=None, stream=None,
                   grad_scale=1.0, grad_f32=False, profile=False, rate=0):
    """(sum of misfits, sum of gradients over shots (FP64, or FP32 with grad_f32), stats dict).

    The shots run as batches of lanes, one launch per stencil step over all
    lanes of a batch."""
    n = len(shots)
    if len(d_obs_list) != n:
        raise ValueError("one d_obs per shot")
    ptrs, mem = _d_obs_ptrs(d_obs_list)
    gdt = np.float32 if grad_f32 else np.float64
    if grad_sum is None:
        grad_sum = _alloc(tuple(grid.shape), gdt, "cuda" if mem == DEVICE else None)
    pg, memg = _buf(grad_sum, gdt)
    if memg != mem:
        raise ValueError("d_obs and grad_sum must both be host or both be device buffers")
    for sh, d in zip(shots, d_obs_list):
        _need(d, (grid.nt + 1) * sh.nrec, "d_obs")
    _need(grad_sum, grid.npts, "grad_sum")
    carr, keep = _shot_array(shots, grid.nt)
    o = _opts(ckpt_slots, store_mode, tol, pool_bytes, grad_kind, use_graph, profile, grad_scale, grad_f32,
              rate=rate)
    phi = ctypes.c_double(0.0)
    st = Stats()
    _check(lib().ckfwi_batch_gradient(model, carr, n, ptrs, mem, ctypes.byref(o), ctypes.byref(phi), pg,
                                      ctypes.byref(st), _stream(stream)), "ckfwi_batch_gradient")
    del keep
    return phi.value, grad_sum, st.as_dict()


def batch_gradient_models(models, shots, d_obs_list, offsets, global_shape, ckpt_slots, store_mode=STORE_FP32,
                          tol=0.0, pool_bytes=0, grad_kind=SLOWNESS2, use_graph=False, grad_sum=None, stream=None,
                          grad_scale=1.0, grad_f32=False, profile=False, rate=0):
    """Shots with uneven apertures: shot s on its own model (window) models[s],
    placed at offsets[s] = (z, y, x) in a global grid of global_shape.
    Returns (sum of misfits, gradient sum on the global grid, stats dict)."""
    n = len(shots)
    if len(models) != n or len(d_obs_list) != n or len(offsets) != n:
        raise ValueError("one model, d_obs and offset per shot")
    ptrs, mem = _d_obs_ptrs(d_obs_list)
    gshape = tuple(int(v) for v in global_shape)
    if len(gshape) == 2:
        gn = (gshape[0], 1, gshape[1])
    else:
        gn = gshape
    gdt = np.float32 if grad_f32 else np.float64
    if grad_sum is None:
        grad_sum = _alloc(gshape, gdt, "cuda" if mem == DEVICE else None)
    pg, memg = _buf(grad_sum, gdt)
    if memg != mem:
        raise ValueError("d_obs and grad_sum must both be host or both be device buffers")
    _need(grad_sum, int(np.prod(gshape)), "grad_sum")
    nt = None
    for m, sh, d in zip(models, shots, d_obs_list):
        if isinstance(m, Model):
            nt = m.grid.nt
            _need(d, (nt + 1) * sh.nrec, "d_obs")
    marr = (ctypes.c_void_p * n)(*[m.h if isinstance(m, Model) else m for m in models])
    off = np.zeros((n, 3), dtype=np.int32)
    for i, o3 in enumerate(offsets):
        o3 = tuple(int(v) for v in o3)
        off[i] = (o3[0], 0, o3[1]) if len(o3) == 2 else o3
    gna = (ctypes.c_int * 3)(*gn)
    carr, keep = _shot_array(shots, nt)
    o = _opts(ckpt_slots, store_mode, tol, pool_bytes, grad_kind, use_graph, profile, grad_scale, grad_f32,
              rate=rate)
    phi = ctypes.c_double(0.0)
    st = Stats()
    _check(lib().ckfwi_batch_gradient_models(marr, carr, n, ptrs, mem, ctypes.byref(o), off.ctypes.data, gna,
                                             ctypes.byref(phi), pg, ctypes.byref(st), _stream(stream)),
           "ckfwi_batch_gradient_models")
    del keep
    return phi.value, grad_sum, st.as_dict()


def free(model):
    if model:
        lib().ckfwi_free(model)


def revolve_schedule(nt, slots):
    """(actions int32 [n][3], (p, W, R)) of the library's Revolve schedule."""
    n = ctypes.c_longlong(0)
    cnt = (ctypes.c_longlong * 3)()
    _check(lib().ckfwi_revolve_schedule(int(nt), int(slots), None, 0, ctypes.byref(n), cnt),
           "ckfwi_revolve_schedule")
    acts = np.zeros((n.value, 3), dtype=np.int32)
    _check(lib().ckfwi_revolve_schedule(int(nt), int(slots), acts.ctypes.data, n.value, ctypes.byref(n), cnt),
           "ckfwi_revolve_schedule")
    return acts, (cnt[0], cnt[1], cnt[2])


def multistage_schedule(nt, slots, host_slots):
    """(actions int32 [n][3], (p, W, R)) of the schedule of a gradient with
    FP32 checkpoints in two storage levels (slots 1 .. host_slots on the host)."""
    n = ctypes.c_longlong(0)
    cnt = (ctypes.c_longlong * 3)()
    args = (int(nt), int(slots), int(host_slots))
    _check(lib().ckfwi_multistage_schedule(*args, None, 0, ctypes.byref(n), cnt), "ckfwi_multistage_schedule")
    acts = np.zeros((n.value, 3), dtype=np.int32)
    _check(lib().ckfwi_multistage_schedule(*args, acts.ctypes.data, n.value, ctypes.byref(n), cnt),
           "ckfwi_multistage_schedule")
    return acts, (cnt[0], cnt[1], cnt[2])


def stream_words(model):
    """Words of every compression of the model's last compressed-checkpoint
    gradient, in schedule order (u^s, u^{s-1} per takeshot)."""
    n = ctypes.c_longlong(0)
    _check(lib().ckfwi_stream_words(model, None, 0, ctypes.byref(n)), "ckfwi_stream_words")
    out = np.zeros(n.value, dtype=np.int64)
    if n.value:
        _check(lib().ckfwi_stream_words(model, out.ctypes.data, n.value, ctypes.byref(n)), "ckfwi_stream_words")
    return out


def codec_bound_words(dims, nz, ny, nx):
    v = lib().ckfwi_codec_bound_words(int(dims), int(nz), int(ny), int(nx))
    if v < 0:
        raise CkfwiError(int(v), "ckfwi_codec_bound_words")
    return int(v)


def _shape3(shape):
    return (shape[0], shape[1], shape[2]) if len(shape) == 3 else (shape[0], 1, shape[1])


def codec_compress(x, tol, stream=None):
    """Compress a contiguous float32 CUDA tensor; returns (int32 tensor holding the
    uint32 stream words, nonfinite flag)."""
    import torch
    if not _is_torch_cuda(x) or x.dtype != torch.float32 or not x.is_contiguous():
        raise ValueError("codec_compress needs a contiguous float32 CUDA tensor")
    dims = x.dim()
    nz, ny, nx = _shape3(tuple(x.shape))
    cap = codec_bound_words(dims, nz, ny, nx)
    out = torch.zeros(cap, dtype=torch.int32, device=x.device)
    used = ctypes.c_longlong(0)
    flags = ctypes.c_int(0)
    with torch.cuda.device(x.device):
        _check(lib().ckfwi_codec_compress(ctypes.c_void_p(x.data_ptr()), dims, nz, ny, nx, float(tol),
                                          ctypes.c_void_p(out.data_ptr()), cap, ctypes.byref(used),
                                          ctypes.byref(flags), _stream(stream)), "ckfwi_codec_compress")
    return out[:used.value].clone(), bool(flags.value & 1)


def codec_compress_noalloc(x, out, tol, stream=None):
    """Allocation-free compression into the caller's int32 CUDA tensor `out`
    (stream words); the library allocates nothing (its scratch is a fixed
    device array, fields up to 65536 blocks).  For callers that cannot let the
    library call cudaMalloc.  Returns (words used, nonfinite flag)."""
    import torch
    if not _is_torch_cuda(x) or x.dtype != torch.float32 or not x.is_contiguous():
        raise ValueError("codec_compress_noalloc needs a contiguous float32 CUDA tensor")
    if not _is_torch_cuda(out) or not out.is_contiguous() or out.element_size() != 4:
        raise ValueError("codec_compress_noalloc needs a contiguous CUDA output tensor of 32-bit words")
    if out.device != x.device:
        raise ValueError("codec_compress_noalloc: x and out must be on the same device")
    dims = x.dim()
    nz, ny, nx = _shape3(tuple(x.shape))
    used = ctypes.c_longlong(0)
    flags = ctypes.c_int(0)
    # the library launches on, and takes its scratch of, the current device
    with torch.cuda.device(x.device):
        _check(lib().ckfwi_codec_compress_noalloc(ctypes.c_void_p(x.data_ptr()), dims, nz, ny, nx, float(tol),
                                                  ctypes.c_void_p(out.data_ptr()), out.numel(), ctypes.byref(used),
                                                  ctypes.byref(flags), _stream(stream)),
               "ckfwi_codec_compress_noalloc")
    return used.value, bool(flags.value & 1)


def codec_rate_words(dims, nz, ny, nx, rate):
    v = lib().ckfwi_codec_rate_words(int(dims), int(nz), int(ny), int(nx), int(rate))
    if v < 0:
        raise CkfwiError(int(v), "ckfwi_codec_rate_words")
    return int(v)


def codec_compress_rate(x, rate, stream=None):
    """Fixed-rate compression (rate bits per value) of a contiguous float32
    CUDA tensor; returns (int32 tensor of stream words, nonfinite flag)."""
    import torch
    if not _is_torch_cuda(x) or x.dtype != torch.float32 or not x.is_contiguous():
        raise ValueError("codec_compress_rate needs a contiguous float32 CUDA tensor")
    dims = x.dim()
    nz, ny, nx = _shape3(tuple(x.shape))
    cap = codec_rate_words(dims, nz, ny, nx, rate)
    out = torch.zeros(cap, dtype=torch.int32, device=x.device)
    used = ctypes.c_longlong(0)
    flags = ctypes.c_int(0)
    _check(lib().ckfwi_codec_compress_rate(ctypes.c_void_p(x.data_ptr()), dims, nz, ny, nx, int(rate),
                                           ctypes.c_void_p(out.data_ptr()), cap, ctypes.byref(used),
                                           ctypes.byref(flags), _stream(stream)), "ckfwi_codec_compress_rate")
    return out[:used.value].clone(), bool(flags.value & 1)


def codec_decompress(stream_words, shape, stream=None):
    import torch
    if not _is_torch_cuda(stream_words) or not stream_words.is_contiguous() or stream_words.element_size() != 4:
        raise ValueError("codec_decompress needs a contiguous CUDA tensor of 32-bit stream words")
    dims = len(shape)
    nz, ny, nx = _shape3(tuple(shape))
    out = torch.zeros(tuple(shape), dtype=torch.float32, device=stream_words.device)
    with torch.cuda.device(stream_words.device):
        _check(lib().ckfwi_codec_decompress(ctypes.c_void_p(stream_words.data_ptr()), stream_words.numel(), dims,
                                            nz, ny, nx, ctypes.c_void_p(out.data_ptr()), _stream(stream)),
               "ckfwi_codec_decompress")
    return out


class Model:
    """Owning wrapper: create_model on construction, free on close / GC."""

    def __init__(self, grid: GridSpec):
        self.grid = grid
        self.h = create_model(grid)

    def set_model(self, data, kind=VELOCITY, stream=None):
        _need(data, self.grid.npts, "the medium")
        set_model(self.h, data, kind, stream)

    def forward_shot(self, shot, **kw):
        return forward_shot(self.h, self.grid, shot, **kw)

    def misfit(self, shot, d_obs, **kw):
        return misfit(self.h, self.grid, shot, d_obs, **kw)

    def adjoint_gradient(self, shot, d_obs, ckpt_slots, **kw):
        return adjoint_gradient(self.h, self.grid, shot, d_obs, ckpt_slots, **kw)

    def stream_words(self):
        return stream_words(self.h)

    def batch_gradient(self, shots, d_obs_list, ckpt_slots, **kw):
        return batch_gradient(self.h, self.grid, shots, d_obs_list, ckpt_slots, **kw)

    def close(self):
        if self.h:
            free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
