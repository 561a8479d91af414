// Device code of the forward and fused reverse time steps of the OT2
// acoustic kernel (Sec. 6, Eq. "eqn:wave"; the recursion and its exact
// transpose are stated in include/ckfwi.h), shared by the single-shot
// kernels (kernels.cu) and the batched ones (batch.cu).
//
// Both kernels are HBM-bound stencils.  A CTA owns a BX x BY column block
// of the (x, y) plane and marches down a run of zlen z planes: the z
// neighbours of each column live in a register queue of 2K+1 values, the
// current plane (with a K-wide x/y halo) is staged in shared memory, and the
// next plane's global loads are issued before the current plane is
// computed.  Every field value is read from HBM once per step (halo reuse
// happens in shared memory and L2); the damping rate is rebuilt from three
// small per-axis tables instead of being streamed.
//
// Rounding: the update is spelled out with __fmaf_rn / __fadd_rn /
// __fdividef in one device function used by every kernel, so no compiler
// contraction can make the forward step of a recomputation differ from the
// first sweep; with compression off, a checkpointed gradient is bitwise the
// store-all gradient.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace ckfwi {

template <class T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }

template <class T> __device__ __forceinline__ float ldf(const T* p) { return to_f<T>(p[0]); }
template <> __device__ __forceinline__ float ldf<float>(const float* p) { return __ldg(p); }

// One leapfrog update with damping, a u' = 2c - b p + w s with a, b = 1 +- e,
// e = eta dt/2, evaluated in increment form:
//   u' = c + ((1 - e)(c - p) + w s) / (1 + e).
// The same recursion, but the only rounding at the scale of |u| is the
// final addition: c - p is nearly exact and the damping factors multiply
// that small increment, so FP32 keeps the receivers about five times closer
// to the FP64 oracle over thousands of steps than 2c - b p + w s would.
// For the same reason the division by 1 + e (inside the damping layer only)
// may be the fast approximate one (2 ulp of the increment): it is one
// reciprocal and one multiply instead of the IEEE division's sequence, and
// every kernel uses the same instruction, so they stay bitwise equal.
__device__ __forceinline__ float leapfrog(float c, float p, float w, float s, float eta, float hdt)
{
    const float be = __fmaf_rn(-eta, hdt, 1.0f);
    float t = __fmaf_rn(w, s, __fmul_rn(be, __fsub_rn(c, p)));
    t = eta != 0.0f ? __fdividef(t, __fmaf_rn(eta, hdt, 1.0f)) : t;
    return __fadd_rn(c, t);
}

struct InjCol {          // per-thread part of an injection test
    bool col;
    int base;            // (y - y0) * (x1 - x0) + (x - x0)
    int plane;           // (y1 - y0) * (x1 - x0)
};

__device__ __forceinline__ InjCol inj_col(const Inj& in, int y, int x, bool act)
{
    InjCol c;
    c.col = act && in.on && y >= in.y0 && y < in.y1 && x >= in.x0 && x < in.x1;
    c.plane = (in.y1 - in.y0) * (in.x1 - in.x0);
    c.base = (y - in.y0) * (in.x1 - in.x0) + (x - in.x0);
    return c;
}

__device__ __forceinline__ float inj_val(const Inj& in, const InjCol& c, int z)
{
    float acc = 0.0f;
    if (c.col && z >= in.z0 && z < in.z1) {
        const int b = (z - in.z0) * c.plane + c.base;
        const int e1 = in.rowptr[b + 1];
        for (int e = in.rowptr[b]; e < e1; ++e) acc = __fmaf_rn(in.wt[e], in.series[in.col[e]], acc);
    }
    return acc;
}

// Laplacian from the register queue (z) and the shared tile (x, y), in
// difference form: sum_j c_j sum_axes ((u_{+j} - u) + (u_{-j} - u)).  The
// differences of neighbouring values are nearly exact, so the large
// cancelling terms c_0 u and sum_j c_j (u_{+j} + u_{-j}) are never formed;
// at order 16 this keeps FP32 receivers within 1e-5 of the FP64 oracle
// where the plain form does not.  Terms are added from j = K down to 1.
template <int K, int DIMS, int SX>
__device__ __forceinline__ float lap_at(const float (&q)[2 * K + 1], const float* sm, int cy, int cx,
                                        const float* c)
{
    const float u = q[K];
    float acc = 0.0f;
#pragma unroll
    for (int j = K; j >= 1; --j) {
        float s = __fadd_rn(__fsub_rn(q[K + j], u), __fsub_rn(q[K - j], u));
        s = __fadd_rn(s, __fadd_rn(__fsub_rn(sm[cy * SX + cx + j], u), __fsub_rn(sm[cy * SX + cx - j], u)));
        if (DIMS == 3)
            s = __fadd_rn(s, __fadd_rn(__fsub_rn(sm[(cy + j) * SX + cx], u), __fsub_rn(sm[(cy - j) * SX + cx], u)));
        acc = __fmaf_rn(c[j], s, acc);
    }
    return acc;
}

// Stage plane values of one field into its shared tile: centre from the
// queue, halos from registers loaded one iteration ahead.
template <int K, int DIMS, int BX, int BY>
struct Halo {
    float xl, xr, yl, yr;
    template <class T>
    __device__ __forceinline__ void load(const T* f, long long zoff, long long col, int tx, int ty,
                                         int x, int y, int nx, int ny, long long px)
    {
        xl = xr = yl = yr = 0.0f;
        if (tx < K && y < ny) {
            xl = ldf<T>(f + zoff + col - K);
            if (x + BX < nx + K) xr = ldf<T>(f + zoff + col + BX);
        }
        if (DIMS == 3 && ty < K && x < nx) {
            yl = ldf<T>(f + zoff + col - (long long)K * px);
            if (y + BY < ny + K) yr = ldf<T>(f + zoff + col + (long long)BY * px);
        }
    }
    __device__ __forceinline__ void store(float* sm, float centre, int tx, int ty) const
    {
        constexpr int SX = BX + 2 * K;
        const int cy = (DIMS == 3) ? ty + K : 0;
        sm[cy * SX + tx + K] = centre;
        if (tx < K) {
            sm[cy * SX + tx] = xl;
            sm[cy * SX + tx + BX + K] = xr;
        }
        if (DIMS == 3 && ty < K) {
            sm[ty * SX + tx + K] = yl;
            sm[(ty + BY + K) * SX + tx + K] = yr;
        }
    }
};

// Body of the forward step for CTA (bx, by, bz) of the step's grid.
// (gxn, gyn: CTAs of the step's grid along x and y.)
template <int K, int DIMS, int BX, int BY, int CK>
__device__ __forceinline__ void fwd_body(const FwdArgs& a, float* sm, int bxi, int byi, int bzi, int gxn, int gyn)
{
    constexpr int SX = BX + 2 * K;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nz = a.g.nz, ny = a.g.ny, nx = a.g.nx;
    const long long px = a.g.px, pxy = a.g.pxy;
    const int x = bxi * BX + tx;
    const int y = (DIMS == 3) ? byi * BY + ty : 0;
    const bool act = (x < nx) && (y < ny);

    // receiver sampling of u^n by the first threads of the grid
    if (a.smp.n > 0) {
        const int gt = ((bzi * gyn + byi) * gxn + bxi) * (BX * BY) + ty * BX + tx;
        if (gt < a.smp.n) {
            float acc = 0.0f;
            for (int i = 0; i < a.smp.nst; ++i)
                acc = __fmaf_rn(a.smp.wt[gt * a.smp.nst + i], __ldg(a.u + a.smp.idx[gt * a.smp.nst + i]), acc);
            a.smp.out[gt] = acc;
        }
    }

    const int z0 = bzi * a.zlen;
    if (z0 >= nz) return;
    const int z1 = min(z0 + a.zlen, nz);
    const long long col = (long long)y * px + x;
    const float ecol = act ? ((DIMS == 3 ? a.eta[nz + y] : 0.0f) + a.eta[nz + ny + x]) : 0.0f;
    const InjCol ic = inj_col(a.src, y, x, act);
    const int cy = (DIMS == 3) ? ty + K : 0;

    float q[2 * K + 1];
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) q[i] = act ? __ldg(a.u + (long long)(z0 - K + i) * pxy + col) : 0.0f;
    float nq = act ? __ldg(a.u + (long long)(z0 + K) * pxy + col) : 0.0f;
    float nup = act ? __ldg(a.up + (long long)z0 * pxy + col) : 0.0f;
    float nw = act ? __ldg(a.w + (long long)z0 * pxy + col) : 0.0f;
    Halo<K, DIMS, BX, BY> hn;
    hn.load(a.u, (long long)z0 * pxy, col, tx, ty, x, y, nx, ny, px);

    for (int z = z0; z < z1; ++z) {
        q[2 * K] = nq;
        const float upv = nup, wv = nw;
        const Halo<K, DIMS, BX, BY> hc = hn;
        if (z + 1 < z1) {
            const long long zo = (long long)(z + 1) * pxy;
            nq = act ? __ldg(a.u + zo + (long long)K * pxy + col) : 0.0f;
            nup = act ? __ldg(a.up + zo + col) : 0.0f;
            nw = act ? __ldg(a.w + zo + col) : 0.0f;
            hn.load(a.u, zo, col, tx, ty, x, y, nx, ny, px);
        }
        __syncthreads();
        hc.store(sm, q[K], tx, ty);
        __syncthreads();
        if (act) {
            float s = lap_at<K, DIMS, SX>(q, sm, cy, tx + K, a.c);
            s = __fadd_rn(s, inj_val(a.src, ic, z));
            const float eta = a.eta[z] + ecol;
            const float v = leapfrog(q[K], upv, wv, s, eta, a.hdt);
            const long long o = (long long)z * pxy + col;
            a.out[o] = v;
            if (CK == CK_FP32) {
                static_cast<float*>(a.ck_up)[o] = q[K];
            } else if (CK == CK_BF16) {
                static_cast<__nv_bfloat16*>(a.ck_u)[o] = __float2bfloat16_rn(v);
                static_cast<__nv_bfloat16*>(a.ck_up)[o] = __float2bfloat16_rn(q[K]);
            } else if (CK == CK_FP16) {
                const __half hv = __float2half_rn(v), hp = __float2half_rn(q[K]);
                static_cast<__half*>(a.ck_u)[o] = hv;
                static_cast<__half*>(a.ck_up)[o] = hp;
                if (__hisinf(hv) || __hisinf(hp)) atomicOr(a.err, 1);
            }
        }
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) q[i] = q[i + 1];
    }
}

// Body of the fused reverse step for CTA (bx, by, bz) of the step's grid.
template <int K, int DIMS, int BX, int BY, class UT>
__device__ __forceinline__ void adj_body(const AdjArgs& a, float* sm, int bxi, int byi, int bzi)
{
    constexpr int SX = BX + 2 * K;
    constexpr int TILE = (DIMS == 3 ? BY + 2 * K : 1) * SX;
    float* sl = sm;
    float* su = sm + TILE;
    const UT* uu = static_cast<const UT*>(a.u);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nz = a.g.nz, ny = a.g.ny, nx = a.g.nx;
    const long long px = a.g.px, pxy = a.g.pxy;
    const int x = bxi * BX + tx;
    const int y = (DIMS == 3) ? byi * BY + ty : 0;
    const bool act = (x < nx) && (y < ny);
    const int z0 = bzi * a.zlen;
    if (z0 >= nz) return;
    const int z1 = min(z0 + a.zlen, nz);
    const long long col = (long long)y * px + x;
    const float ecol = act ? ((DIMS == 3 ? a.eta[nz + y] : 0.0f) + a.eta[nz + ny + x]) : 0.0f;
    const InjCol ia = inj_col(a.adj, y, x, act);
    const InjCol is = inj_col(a.src, y, x, act);
    const int cy = (DIMS == 3) ? ty + K : 0;

    float ql[2 * K + 1], qu[2 * K + 1];
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) {
        const long long o = (long long)(z0 - K + i) * pxy + col;
        ql[i] = act ? __ldg(a.l1 + o) : 0.0f;
        qu[i] = act ? ldf<UT>(uu + o) : 0.0f;
    }
    long long o0 = (long long)(z0 + K) * pxy + col;
    float nql = act ? __ldg(a.l1 + o0) : 0.0f;
    float nqu = act ? ldf<UT>(uu + o0) : 0.0f;
    o0 = (long long)z0 * pxy + col;
    float nl2 = act ? __ldg(a.l2 + o0) : 0.0f;
    float nw = act ? __ldg(a.w + o0) : 0.0f;
    float ng = act ? a.gacc[o0] : 0.0f;
    Halo<K, DIMS, BX, BY> hln, hun;
    hln.load(a.l1, (long long)z0 * pxy, col, tx, ty, x, y, nx, ny, px);
    hun.load(uu, (long long)z0 * pxy, col, tx, ty, x, y, nx, ny, px);

    for (int z = z0; z < z1; ++z) {
        ql[2 * K] = nql;
        qu[2 * K] = nqu;
        const float l2v = nl2, wv = nw, gv = ng;
        const Halo<K, DIMS, BX, BY> hlc = hln, huc = hun;
        if (z + 1 < z1) {
            const long long zo = (long long)(z + 1) * pxy;
            nql = act ? __ldg(a.l1 + zo + (long long)K * pxy + col) : 0.0f;
            nqu = act ? ldf<UT>(uu + zo + (long long)K * pxy + col) : 0.0f;
            nl2 = act ? __ldg(a.l2 + zo + col) : 0.0f;
            nw = act ? __ldg(a.w + zo + col) : 0.0f;
            ng = act ? a.gacc[zo + col] : 0.0f;
            hln.load(a.l1, zo, col, tx, ty, x, y, nx, ny, px);
            hun.load(uu, zo, col, tx, ty, x, y, nx, ny, px);
        }
        __syncthreads();
        hlc.store(sl, ql[K], tx, ty);
        huc.store(su, qu[K], tx, ty);
        __syncthreads();
        if (act) {
            float sl_ = lap_at<K, DIMS, SX>(ql, sl, cy, tx + K, a.c);
            sl_ = __fadd_rn(sl_, inj_val(a.adj, ia, z));
            float su_ = lap_at<K, DIMS, SX>(qu, su, cy, tx + K, a.c);
            su_ = __fadd_rn(su_, inj_val(a.src, is, z));
            const float eta = a.eta[z] + ecol;
            const float lam = leapfrog(ql[K], l2v, wv, sl_, eta, a.hdt);
            const long long o = (long long)z * pxy + col;
            a.l0[o] = lam;
            a.gacc[o] = __fmaf_rn(lam, su_, gv);
        }
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) {
            ql[i] = ql[i + 1];
            qu[i] = qu[i + 1];
        }
    }
}


// dynamic shared memory of a step: `fields` staged planes with x / y halos
template <int DIMS, int BX, int BY>
inline size_t smem_bytes(int K, int fields)
{
    return (size_t)fields * (DIMS == 3 ? BY + 2 * K : 1) * (BX + 2 * K) * sizeof(float);
}

// Batched launches: lane l owns CTAs start[l] .. start[l+1]-1 of a 1D grid;
// each CTA finds its lane by binary search and stages the lane's argument
// block in shared memory.  Returns the CTA's index inside its lane.
__device__ __forceinline__ int lane_of(const int* __restrict__ start, int nl, int b)
{
    int lo = 0, hi = nl - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(start + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <class Args>
__device__ __forceinline__ int stage_args(Args& dst, const Args* __restrict__ tab, const int* __restrict__ start,
                                          int nl)
{
    static_assert(sizeof(Args) % 4 == 0, "argument block must be whole words");
    const int l = lane_of(start, nl, blockIdx.x);
    const int* src = reinterpret_cast<const int*>(tab + l);
    int* d = reinterpret_cast<int*>(&dst);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int i = tid; i < (int)(sizeof(Args) / 4); i += blockDim.x * blockDim.y) d[i] = __ldg(src + i);
    __syncthreads();
    return blockIdx.x - __ldg(start + l);
}

}  // namespace ckfwi
