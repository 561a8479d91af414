/*
 * ckfwi — checkpointed, compressed adjoint-state gradients of acoustic
 * seismic inversion on one GB300 (sm_103a).
 *
 * Method: Kukreja, Hueckelheim, Louboutin, Hovland, Gorman, "Combining
 * checkpointing and data compression to accelerate adjoint-based
 * optimization problems" (arXiv 1810.05268).
 *   Sec. 6, Eq. "eqn:wave":  m u_tt - lap(u) = q, m = 1/c^2; the misfit
 *     phi = 1/2 ||d_sim - d_obs||^2 and its gradient by the adjoint-state
 *     method with the OT2 (2nd order in time) kernel.
 *   Sec. 3, Eq. "eqn:recompute":  Revolve binomial checkpointing with M
 *     slots; checkpoints copied between working and checkpoint memory.
 *   Sec. 2.2 and Sec. 4:  checkpoints stored compressed (typecast or a
 *     fixed-tolerance lossy codec), giving F times more slots at equal memory.
 *
 * Discretisation (the paper leaves it to its DSL; this library fixes it):
 *   a u^{n+1} = 2 u^n - b u^{n-1} + w (lap_h u^n + Q^T s^n), n = 0..N-1,
 *   u^0 = u^-1 = 0, w = dt^2 c^2, a = 1 + eta dt/2, b = 1 - eta dt/2, with
 *   lap_h the 2k-th order central Laplacian (k = space_order/2, zero values
 *   outside the total grid) and eta the damping rate of the absorbing layer,
 *   sum over axes of eta_max (delta/L)^2, L = nbl h,
 *   eta_max = 3 vmax_damp/(2L) ln(1/R), R = 1e-3.
 *   Sources and receivers use multilinear weights over the 2^d surrounding
 *   grid points; d^n = P u^n for n = 0..N (d^0 = 0); the misfit sums
 *   n = 1..N.  The adjoint is the exact transpose of this recursion; the
 *   gradient is dphi/dm = sum_{n=0}^{N-1} lam^n (lap_h u^n + Q^T s^n) c^2.
 *
 * OT4 kernel (Sec. 6: the 4th-order-in-time kernel the paper takes from its
 * DSL without stating it; time_order = 4).  The recursion above with lap_h
 * replaced by
 *   A u = lap_h u + dt^2/12 lap_h(c^2 lap_h u),
 * the modified-equation correction of the leapfrog's dt^2/12 u_tttt error
 * (the inner field c^2 lap_h u is zero outside the total grid, like u);
 * damping and sources enter as for OT2.  A is symmetric, so the adjoint is
 * the same recursion with A, and the exact gradient gains the derivative of
 * the correction with respect to m:
 *   dphi/dm = sum_{n=0}^{N-1} [ lam^n (A u^n + Q^T s^n) c^2
 *                              + dt^2/12 c^4 (lap_h u^n)(lap_h lam^n) ].
 * A step costs two launches; a model of time order 4 computes the gradients
 * of a batch one shot at a time.
 *
 * Units: lengths in m, times in ms, velocities in km/s (= m/ms), m = 1/c^2.
 *
 * Arrays: velocity, slowness and gradient fields cover the total grid
 * (interior + damping layer), dense, [nz][ny][nx] with x fastest (2D:
 * [nz][nx]).  Trace arrays are [nt+1][nrec].  A `mem` argument says where a
 * caller buffer lives: CKFWI_HOST (pageable or pinned host memory; the call
 * copies through its own device buffers and synchronises the stream) or
 * CKFWI_DEVICE (device memory on the current device; the call is
 * asynchronous on `stream` except where noted).  The caller owns every
 * buffer it passes; the model owns its working fields, checkpoint pool and
 * maps, all released by ckfwi_free.  `stream` is a cudaStream_t (NULL = the
 * legacy default stream).
 *
 * Errors: every int-returning function returns CKFWI_OK (0) or a negative
 * status below; outputs are unspecified after an error; nothing aborts and
 * no C++ exception crosses this boundary.  A model is used by one host
 * thread at a time.
 */
#ifndef CKFWI_H
#define CKFWI_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CKFWI_API __attribute__((visibility("default")))
#else
#define CKFWI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define CKFWI_OK 0
#define CKFWI_EINVAL -1         /* bad argument, geometry or size */
#define CKFWI_ENOMEM -2         /* device or host allocation failed */
#define CKFWI_POOL_OVERFLOW -3  /* compressed checkpoints exceeded the pool */
#define CKFWI_NONFINITE -4      /* NaN/Inf met, or FP16 checkpoint overflow */
#define CKFWI_CORRUPT -5        /* compressed stream failed its checks */
#define CKFWI_TIMEOUT -6        /* a bounded device wait gave up */
#define CKFWI_ECUDA -7          /* a CUDA runtime call failed */

#define CKFWI_HOST 0
#define CKFWI_DEVICE 1

/* checkpoint storage (Sec. 2: a typecast is a lossy compressor of ratio 2;
 * CODEC is the fixed-tolerance block codec, Sec. 2.2) */
#define CKFWI_STORE_FP32 0
#define CKFWI_STORE_BF16 1
#define CKFWI_STORE_FP16 2
#define CKFWI_STORE_CODEC 3
/* the codec's fixed-rate mode (Sec. 2.2 lists ZFP's fixed-rate mode: a
 * guaranteed size, no error bound): `rate` bits per value, every checkpoint
 * the same predictable size (ckfwi_codec_rate_words) */
#define CKFWI_STORE_CODEC_RATE 4

/* model parameterisation of set_model / of the gradient */
#define CKFWI_VELOCITY 0   /* c [km/s]; gradient dphi/dc */
#define CKFWI_SLOWNESS2 1  /* m = 1/c^2 [ms^2/m^2]; gradient dphi/dm */

typedef struct ckfwi_grid {
    int dims;            /* 2 or 3 */
    int n[3];            /* total grid incl. damping layer: nz, ny, nx (ny = 1 in 2D) */
    int nbl;             /* damping-layer width [cells] on every face, >= 0 */
    double h;            /* grid spacing [m] */
    int space_order;     /* 2, 4, 8 or 16 */
    double dt;           /* time step [ms] */
    int nt;              /* number of time steps N >= 1 */
    double vmax_damp;    /* largest velocity the model will hold [km/s]: sets the
                            damping strength and the stability check */
    int time_order;      /* 2: OT2 kernel (0 reads as 2); 4: OT4 kernel */
} ckfwi_grid;

typedef struct ckfwi_shot {
    double src[3];       /* source position (z, y, x) [m] from the first interior
                            point; 2D ignores y */
    double f0;           /* Ricker peak frequency [kHz] */
    double t0;           /* Ricker delay [ms]; <= 0 selects 1.5/f0 */
    double amp;          /* Ricker amplitude */
    const float* wavelet;/* optional host array [nt]: source time function used
                            instead of the Ricker wavelet */
    int nrec;            /* number of receivers >= 1 */
    const double* rec;   /* host [nrec][3] receiver positions (z, y, x) [m] */
} ckfwi_shot;

typedef struct ckfwi_grad_opts {
    int ckpt_slots;      /* M: checkpoint slots incl. the initial state, >= 1;
                            M >= nt selects store-all (every state kept) */
    int store_mode;      /* CKFWI_STORE_* */
    double tol;          /* CODEC: absolute point-wise bound (> 0, >= 2^-90) */
    size_t pool_bytes;   /* CODEC: byte budget of the checkpoint pool;
                            0 = (M-1) uncompressed states */
    int grad_kind;       /* CKFWI_VELOCITY or CKFWI_SLOWNESS2 */
    int use_graph;       /* 1: record the gradient as a CUDA graph on the first
                            call with this configuration and replay it after */
    int profile;         /* 1: time every kernel class with CUDA events on the
                            stream (fills the *_ms fields of ckfwi_stats); not
                            combined with use_graph */
    double grad_scale;   /* the gradient is multiplied by this (0 is read as 1) */
    int grad_f32;        /* batch only: grad_sum is float32 (the FP64 compensated
                            sum rounded once) instead of float64 */
    int host_slots;      /* FP32 / BF16 / FP16 Revolve: how many of the M - 1
                            checkpoint slots live in pinned host memory (the
                            second storage level).  FP32: the gradient follows
                            ckfwi_multistage_schedule (host checkpoints written
                            once, in the first sweep); a host checkpoint goes
                            through a device staging pair and a copy stream,
                            overlapped with the steps, and a host restore is
                            copied ahead of use.  BF16 / FP16: the Revolve
                            schedule, its lowest-numbered slots (written and
                            read least) on the host, read and written by the
                            step kernels over the host link.  0: every slot in
                            device memory.  Values are unchanged by the
                            placement (FP32 checkpoints are exact). */
    int rate;            /* CODEC_RATE: bits per value, 1..32.  The pool holds
                            exactly (M - 1) * 2 fixed-size streams; a non-zero
                            pool_bytes below that is EINVAL. */
} ckfwi_grad_opts;

typedef struct ckfwi_stats {
    long long fwd_steps;     /* forward (advance) steps, incl. the extra step to N */
    long long adj_steps;     /* reverse steps (= nt) */
    long long p;             /* Revolve advance count p(N, M) */
    long long takeshots;     /* W */
    long long restores;      /* R */
    long long kernel_launches;
    double pool_bytes_peak;  /* device bytes of checkpoint storage in use, peak */
    double ratio_min;        /* CODEC: smallest and mean compression ratio */
    double ratio_mean;
    double u_absmax;         /* max |u^N| over the total grid, from a device
                                reduction at the end of the first sweep: the
                                wavefield's scale, against which an absolute
                                codec tolerance (Sec. 2.2) can be read as
                                tol / max|u|.  Batches: the largest over all
                                shots. */
    /* with opts->profile: device time [ms] and launches per kernel class */
    double fwd_ms, adj_ms, comp_ms, decomp_ms, other_ms;
    long long fwd_launches, adj_launches, comp_calls, decomp_calls;
    /* stencil kernel generation the autotuner chose for the forward and the
     * reverse step: 1 register-queue, 2 TMA-fed, 3 vector-blocked, 4 fed by
     * asynchronous copies, 5 / 6 the OT4 kernels (register-queue / vector-
     * blocked), 7 lean asynchronous copies, 8 fed by tensor copies (its
     * reverse step split in two launches); and the tile (x points, y rows,
     * x points per thread, z planes per CTA or, for generation 2, CTAs per
     * SM) */
    int fwd_ver, fwd_bx, fwd_by, fwd_vec, fwd_zlen;
    int adj_ver, adj_bx, adj_by, adj_vec, adj_zlen;
    int fwd_pf, adj_pf;      /* generations 4 and 8: planes of prefetch (4: 0 = the
                                default, 2; 8: 0 reads as 1); generation 7: planes
                                a step (1 or 2) */
} ckfwi_stats;

typedef struct ckfwi_model ckfwi_model;

/* Allocate a model for grid g on the current device (working fields, maps,
 * coefficient buffers).  Sec. 6 (Eq. "eqn:wave").  *out receives the handle.
 * EINVAL for an unsupported space or time order, a non-positive size, a
 * damping layer wider than half the grid, or vmax_damp dt / h beyond the
 * leapfrog stability limit of the stencil (OT4: sqrt(3) times the OT2
 * limit); ENOMEM if device memory runs out. */
CKFWI_API int ckfwi_create_model(const ckfwi_grid* g, ckfwi_model** out);

/* Set the medium: data is c [km/s] (kind CKFWI_VELOCITY) or m = 1/c^2
 * (CKFWI_SLOWNESS2) on the total grid, float32, dense.  Builds the
 * per-point coefficient w = dt^2 c^2 (Sec. 6: m = 1/c^2).  Synchronous.
 * EINVAL for a non-positive or non-finite value (NONFINITE for NaN/Inf). */
CKFWI_API int ckfwi_set_model(ckfwi_model* m, const float* data, int kind, int mem, void* stream);

/* Forward modelling of one shot (Sec. 6, the forward problem): writes
 * d_sim [nt+1][nrec] float32 (row 0 = P u^0 = 0).  Synchronous: it reads
 * the kernels' error flags at the end (TIMEOUT when a TMA kernel's bounded
 * wait ran out).  EINVAL for a source or receiver outside the grid or
 * nrec < 1. */
CKFWI_API int ckfwi_forward_shot(ckfwi_model* m, const ckfwi_shot* s, float* d_sim, int mem, void* stream);

/* Misfit of one shot without its gradient (Sec. 6): forward modelling, the
 * residual and phi = 1/2 sum_{n=1..N} ||d^n - d_obs^n||^2 in FP64 on the
 * device; *misfit (host) receives phi, d_sim (optional, same `mem`) the
 * simulated data.  Synchronous; TIMEOUT as for ckfwi_forward_shot. */
CKFWI_API int ckfwi_misfit(ckfwi_model* m, const ckfwi_shot* s, const float* d_obs, int mem, double* misfit,
                           float* d_sim, void* stream);

/* Misfit and adjoint-state gradient of one shot (Sec. 6), with Revolve
 * checkpointing of M slots (Sec. 3) and optionally compressed checkpoints
 * (Sec. 4).  d_obs [nt+1][nrec] float32 (row 0 ignored); grad receives the
 * gradient on the total grid (dense float32), w.r.t. velocity or m per
 * opts->grad_kind; *misfit (host) receives phi in FP64; stats (optional,
 * host) receives the counters.  Synchronises the stream before returning
 * (the misfit and error flags are read back).  POOL_OVERFLOW if compressed
 * checkpoints outgrow pool_bytes; NONFINITE for NaN/Inf in a checkpoint;
 * CORRUPT if a stored stream fails its checks; TIMEOUT if a TMA kernel's
 * bounded plane wait gave up. */
CKFWI_API int ckfwi_adjoint_gradient(ckfwi_model* m, const ckfwi_shot* s, const float* d_obs, int mem,
                           const ckfwi_grad_opts* opts, double* misfit, float* grad,
                           ckfwi_stats* stats, void* stream);

/* Several shots on one model (Sec. 1.2: shots are independent and their
 * gradients and misfits are summed).  The shots run in batches of B lanes:
 * every lane holds one shot's wavefields, adjoint fields and checkpoint
 * storage, all lanes follow one Revolve schedule, and every forward or
 * reverse step is one kernel launch over the tiles of all lanes (recorded
 * as one CUDA graph when opts->use_graph).  B = min(nshots, free device
 * memory / lane size, CKFWI_MAX_LANES from the environment, default 64);
 * the extra lanes are clones of the model that it owns and keeps.
 * d_obs: nshots arrays [nt+1][nrec_s]; misfit_sum (host, FP64) and grad_sum
 * (dense total grid, same `mem`; float64, or float32 when opts->grad_f32)
 * receive the sums over shots in shot order, accumulated with compensated
 * FP64 summation and multiplied by opts->grad_scale (0 = 1).  Every shot's
 * result is bitwise the one ckfwi_adjoint_gradient computes for it.
 * stats: step counters summed over shots; ratio fields are 0. */
CKFWI_API int ckfwi_batch_gradient(ckfwi_model* m, const ckfwi_shot* shots, int nshots,
                         const float* const* d_obs, int mem, const ckfwi_grad_opts* opts,
                         double* misfit_sum, double* grad_sum, ckfwi_stats* stats,
                         void* stream);

/* A batch of shots with uneven apertures: shot s runs on its own model
 * models[s] (a window of a larger survey model, with its own grid size and
 * medium), all models distinct and sharing dims, space_order and nt.  One
 * Revolve schedule drives every lane and each forward or reverse step is one
 * launch over all windows' tiles, as in ckfwi_batch_gradient.  offsets
 * [nshots][3] (host) place each window's total grid (z, y, x) inside the
 * global grid global_n[3] (host; 2D: y offset 0 and global_n[1] = 1);
 * grad_sum (dense global grid, same `mem`, float64 or float32 per
 * opts->grad_f32) receives sum_s of shot s's gradient added at its window,
 * in shot order with compensated FP64 summation, points outside every
 * window 0; misfit_sum (host) the FP64 sum of the misfits.  EINVAL when a
 * window leaves the global grid, a model repeats or lacks a medium, or a
 * model of time order 4 is one of several shots (the OT4 kernels have no
 * batched form).
 * All lanes run at once: ENOMEM when their storage does not fit. */
CKFWI_API int ckfwi_batch_gradient_models(ckfwi_model* const* models, const ckfwi_shot* shots, int nshots,
                         const float* const* d_obs, int mem, const ckfwi_grad_opts* opts,
                         const int* offsets, const int* global_n, double* misfit_sum,
                         double* grad_sum, ckfwi_stats* stats, void* stream);

/* Release the model and everything it owns (working fields, checkpoint
 * pools, maps, recorded graphs, batch clones); NULL is ignored.  The caller
 * makes sure no work queued on the model is still running. */
CKFWI_API void ckfwi_free(ckfwi_model* m);

/* A static, human-readable text for a status code ("unknown status" for a
 * code this header does not define).  Host only. */
CKFWI_API const char* ckfwi_error_string(int status);

/* Stream lengths [words] of every compression of the model's last
 * ckfwi_adjoint_gradient with compressed (CODEC / CODEC_RATE) checkpoints,
 * in schedule order: two per takeshot, u^s then u^{s-1}.  The sizes the
 * time model and the slot planner need when compression ratios vary from
 * step to step (Sec. 8: non-uniform ratios).  *n (host) receives the count;
 * cap = 0 only queries it; EINVAL if 0 < cap < count.  Host only. */
CKFWI_API int ckfwi_stream_words(const ckfwi_model* m, long long* words, long long cap, long long* n);

/* The Revolve schedule for (nt, slots) (Sec. 3, Eq. "eqn:recompute", split
 * at the smallest minimiser), as int32 triples (op, a, b):
 * 0 = advance(from state a, b steps), 1 = takeshot(state a, slot b),
 * 2 = restore(state a, slot b), 3 = youturn(state a).  Host only; writes at
 * most cap triples, *n_triples receives the full count, counts (optional)
 * receives {p, W, R}.  EINVAL if cap is too small (n_triples still set). */
CKFWI_API int ckfwi_revolve_schedule(int nt, int slots, int32_t* actions, long long cap,
                           long long* n_triples, long long* counts);

/* The schedule of a gradient whose FP32 checkpoints use two storage levels
 * (multi-level checkpointing, a future-work item of Sec. 8, in the
 * multistage form of Stumm and Walther that Sec. 3's model builds on):
 * slots 1 .. host_slots are in host memory, host_slots + 1 .. slots - 1 on
 * the device.  Host checkpoints are taken once each, in the first forward
 * sweep, at the starts of segments; each segment is reversed, last first,
 * by Revolve from its start with the device slots.  The segments give the
 * fewest forward steps within that family (the first sweep's segments are
 * of equal length, since p(n, m) is convex in n; the last one, which the
 * first sweep does not cross, may be longer), ties going to fewer host
 * checkpoints.  host_slots = 0 is ckfwi_revolve_schedule.  Same output
 * convention; EINVAL unless 0 <= host_slots <= slots - 1.  Host only. */
CKFWI_API int ckfwi_multistage_schedule(int nt, int slots, int host_slots, int32_t* actions, long long cap,
                                        long long* n_triples, long long* counts);

/* Fixed-accuracy block codec on dense device fields (Sec. 2.2: ZFP's
 * fixed-tolerance mode is the lossy compressor the paper uses; this codec
 * is a member of the same family, specified in codec.cu).
 * ckfwi_codec_bound_words: words a stream of that shape can need.
 * ckfwi_codec_compress: x (device, float32 dense [nz][ny][nx]) -> out
 *   (device uint32, cap words); *used_words (host) receives the stream
 *   length; *flags (host) bit0 = NONFINITE.  Synchronous.  Uses scratch
 *   memory the library allocates and keeps per device.  POOL_OVERFLOW if
 *   cap is too small.
 * ckfwi_codec_decompress: stream (device) -> x (device).  Synchronous;
 *   CORRUPT if a check fails. */
CKFWI_API long long ckfwi_codec_bound_words(int dims, int nz, int ny, int nx);
/* Fixed-rate mode of the same codec (Sec. 2.2: ZFP's fixed-rate mode): rate
 * bits per value, 1..32, every 4^d block exactly ceil(rate 4^d / 32) words.
 * ckfwi_codec_rate_words: the stream length, 16 + nblocks * that (EINVAL for
 *   a bad shape or rate).
 * ckfwi_codec_compress_rate: as ckfwi_codec_compress (device buffers,
 *   synchronous, *used_words and *flags on the host); POOL_OVERFLOW if cap
 *   is below ckfwi_codec_rate_words.  No scratch memory.
 * ckfwi_codec_decompress reads either mode's streams. */
CKFWI_API long long ckfwi_codec_rate_words(int dims, int nz, int ny, int nx, int rate);
CKFWI_API int ckfwi_codec_compress_rate(const float* x, int dims, int nz, int ny, int nx, int rate,
                              uint32_t* out, long long cap, long long* used_words, int* flags,
                              void* stream);
CKFWI_API int ckfwi_codec_compress(const float* x, int dims, int nz, int ny, int nx, double tol,
                         uint32_t* out, long long cap, long long* used_words, int* flags,
                         void* stream);
CKFWI_API int ckfwi_codec_decompress(const uint32_t* in, long long nwords, int dims, int nz, int ny,
                           int nx, float* x, void* stream);

/* Allocation-free ckfwi_codec_compress, for callers that cannot let the
 * library call cudaMalloc (latency-critical code that must not take its
 * implicit synchronisation, or processes whose device memory belongs to
 * another allocator).  No counterpart in the paper.  Same arguments and
 * output as ckfwi_codec_compress; its scratch is a statically sized device
 * array inside the library (about 17 MB per device, held until exit), so
 * fields are limited to 65536 blocks of 4^d values (EINVAL beyond that).
 * The first call on a device looks up that array's address and should come
 * before any stream capture.  All calls share the array: calls that overlap
 * on the GPU race, so order them on one stream.  Synchronous. */
CKFWI_API int ckfwi_codec_compress_noalloc(const float* x, int dims, int nz, int ny, int nx, double tol,
                                           uint32_t* out, long long cap, long long* used_words,
                                           int* flags, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CKFWI_H */
