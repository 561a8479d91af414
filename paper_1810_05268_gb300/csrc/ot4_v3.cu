// Vector-blocked OT4 kernels for 3D grids: the passes of ot4.cu (Z = w lap f,
// the update with w A f = Z + w lap(Z) / 12, and the reverse step's
// gradient pass with its deferred term) on the thread layout of the
// vector-blocked OT2 kernels (stencil_v3.cuh): a thread owns V consecutive x
// points, global accesses are V-wide vectors, staged planes are double
// buffered with one barrier per plane, and the arithmetic runs on pairs of
// points with packed FP32x2 instructions whose lanes round like the scalar
// operations.  Same operands, same order: every value is bitwise the one
// the register-queue OT4 kernels compute, so the two generations mix freely
// inside one gradient.
#include "stencil_v3.cuh"

namespace ckfwi {
namespace {

// One field staged plane by plane down the CTA's z run (queue of 2K + 1
// vectors, halo values one plane ahead).
template <int K, int V, int TX, int TY, class T>
struct VStage {
    float q[2 * K + 1][V];
    float nq[V];
    HaloVals<K, V, TX, TY> hv;

    __device__ __forceinline__ void start(const T* __restrict__ f, int col, int z0, int pxy, bool cload,
                                          const HaloMap<K, V, TX, TY>& hm, float* sm, int tx, int ty)
    {
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) {
            if (cload) gldu<T, V>(q[i], f + col + (z0 - K + i) * pxy);
            else vzero<V>(q[i]);
        }
        if (cload) gldu<T, V>(nq, f + col + (z0 + K) * pxy);
        else vzero<V>(nq);
        hv.zero();
        hv.load(f, z0 * pxy, hm);
        hv.store(sm, q[K], tx, ty, hm);
    }
    __device__ __forceinline__ void take()
    {
#pragma unroll
        for (int i = 0; i < V; ++i) q[2 * K][i] = nq[i];
    }
    // the queue's next plane (offset zq) and the halo of the next staged plane (offset zn)
    __device__ __forceinline__ void fetch(const T* __restrict__ f, int col, int zq, int zn, bool cload,
                                          const HaloMap<K, V, TX, TY>& hm)
    {
        if (cload) gldu<T, V>(nq, f + col + zq);
        hv.load(f, zn, hm);
    }
    __device__ __forceinline__ void stage(float* sm, int tx, int ty, const HaloMap<K, V, TX, TY>& hm) const
    {
        hv.store(sm, q[K + 1], tx, ty, hm);
    }
    __device__ __forceinline__ void shift()
    {
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) {
#pragma unroll
            for (int k = 0; k < V; ++k) q[i][k] = q[i + 1][k];
        }
    }
};

// leapfrog4() for a pair of points: c + ((1 - e)(c - p) + Z + w s) / (1 + e).
// The product (1 - e)(c - p) is formed with the scalar __fmul_rn, which is
// never merged into a multiply-add: the packed multiply feeding the packed
// addition of Z was contracted into one FFMA2, whose single rounding differs
// from the two of the scalar kernels inside the damping layer (1 - e != 1).
__device__ __forceinline__ float2 leap4v(float2 c, float2 p, float2 w, float2 zc, float2 s, float2 eta, float hdt)
{
    const float2 be = __ffma2_rn(f2(-eta.x, -eta.y), f2(hdt, hdt), f2(1.0f, 1.0f));
    const float2 d = __ffma2_rn(p, f2(-1.0f, -1.0f), c);
    const float2 bd = f2(__fmul_rn(be.x, d.x), __fmul_rn(be.y, d.y));
    float2 t = __ffma2_rn(w, s, __fadd2_rn(zc, bd));
    t.x = eta.x != 0.0f ? __fdividef(t.x, __fmaf_rn(eta.x, hdt, 1.0f)) : t.x;
    t.y = eta.y != 0.0f ? __fdividef(t.y, __fmaf_rn(eta.y, hdt, 1.0f)) : t.y;
    return __fadd2_rn(c, t);
}

// store V values at offset o of a row whose first vector point is x0
template <int V>
__device__ __forceinline__ void vput(float* p, long long o, const float (&v)[V], bool full, int x0, int nx)
{
    if (full) {
        vst<V>(p + o, v);
    } else {
#pragma unroll
        for (int i = 0; i < V; ++i)
            if (x0 + i < nx) p[o + i] = v[i];
    }
}

// Common per-thread geometry of a vector-blocked step.
struct Pos3 {
    int tx, ty, nz, ny, nx, px, pxy, x0, y, col, xb;
    bool rowact, cload, full;
};

template <int V, int TX, int TY, int BXP>
__device__ __forceinline__ Pos3 pos3(const FieldGeom& g)
{
    Pos3 p;
    p.tx = threadIdx.x;
    p.ty = threadIdx.y;
    p.nz = g.nz;
    p.ny = g.ny;
    p.nx = g.nx;
    p.px = (int)g.px;
    p.pxy = (int)g.pxy;
    p.xb = blockIdx.x * BXP;
    p.x0 = p.xb + V * p.tx;
    p.y = blockIdx.y * TY + p.ty;
    p.rowact = p.y < p.ny;
    p.cload = p.rowact && p.x0 < p.nx;
    p.full = p.rowact && p.x0 + V <= p.nx;
    p.col = p.y * p.px + p.x0;
    return p;
}

// ------------------------------------------------------------- pass 1
template <int K, int V, int TX, int TY, int NF, class UT>
__global__ void __launch_bounds__(TX * TY) ot4v_lap_kernel(const Ot4LapArgs a)
{
    using G = G3<K, V, TX, TY>;
    extern __shared__ __align__(16) float smem4[];
    const Pos3 P = pos3<V, TX, TY, G::BXP>(a.g);
    if (a.smp.n > 0) {
        const int gt = ((blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * (TX * TY) + P.ty * TX + P.tx;
        if (gt < a.smp.n) {
            float acc = 0.0f;
            for (int i = 0; i < a.smp.nst; ++i)
                acc = __fmaf_rn(a.smp.wt[gt * a.smp.nst + i], __ldg(a.f0 + a.smp.idx[gt * a.smp.nst + i]), acc);
            a.smp.out[gt] = acc;
        }
    }
    const int z0 = blockIdx.z * a.zlen;
    if (z0 >= P.nz) return;
    const int z1 = min(z0 + a.zlen, P.nz);
    HaloMap<K, V, TX, TY> hm;
    hm.init(P.tx, P.ty, P.xb, P.x0, P.y, P.nx, P.ny, P.px);
    const UT* f1 = static_cast<const UT*>(a.f1);
    const float* __restrict__ W = a.w + P.col;
    VStage<K, V, TX, TY, float> s0;
    VStage<K, V, TX, TY, UT> s1;
    s0.start(a.f0, P.col, z0, P.pxy, P.cload, hm, smem4, P.tx, P.ty);
    if (NF == 2) s1.start(f1, P.col, z0, P.pxy, P.cload, hm, smem4 + G::TILE, P.tx, P.ty);
    float nw[V];
    if (P.cload) gld<V>(nw, W + z0 * P.pxy);
    else vzero<V>(nw);
    const int zqmax = P.nz + K - 1;
    for (int z = z0; z < z1; ++z) {
        float* sm = smem4 + ((z - z0) & 1) * (NF * G::TILE);
        float* smn = smem4 + (((z - z0) & 1) ^ 1) * (NF * G::TILE);
        s0.take();
        if (NF == 2) s1.take();
        float wv[V];
#pragma unroll
        for (int i = 0; i < V; ++i) wv[i] = nw[i];
        const int zn = min(z + 1, z1 - 1) * P.pxy, zq = min(z + K + 1, zqmax) * P.pxy;
        s0.fetch(a.f0, P.col, zq, zn, P.cload, hm);
        if (NF == 2) s1.fetch(f1, P.col, zq, zn, P.cload, hm);
        if (P.cload) gld<V>(nw, W + zn);
        __syncthreads();
        if (P.cload) {
            const long long o = (long long)z * P.pxy + P.col;
            float l[V], r[V];
            lap3<K, V, TX, TY>(l, s0.q, sm, P.tx, P.ty, a.c);
#pragma unroll
            for (int p = 0; p < V / 2; ++p) {
                const float2 t = __fmul2_rn(f2(wv[2 * p], wv[2 * p + 1]), f2(l[2 * p], l[2 * p + 1]));
                r[2 * p] = t.x;
                r[2 * p + 1] = t.y;
            }
            vput<V>(a.z0, o, r, P.full, P.x0, P.nx);
            if (NF == 2) {
                lap3<K, V, TX, TY>(l, s1.q, sm + G::TILE, P.tx, P.ty, a.c);
#pragma unroll
                for (int p = 0; p < V / 2; ++p) {
                    const float2 t = __fmul2_rn(f2(wv[2 * p], wv[2 * p + 1]), f2(l[2 * p], l[2 * p + 1]));
                    r[2 * p] = t.x;
                    r[2 * p + 1] = t.y;
                }
                vput<V>(a.z1, o, r, P.full, P.x0, P.nx);
                if (a.zu_next) {   // the deferred gradient term of the step before: Z_u(j+1) lap(lam^j)/12
                    float d[V], zn[V], gv[V];
                    lap3<K, V, TX, TY>(d, s0.q, sm, P.tx, P.ty, a.c12);
                    const long long oc = P.col + (long long)z * P.pxy;
                    if (P.full) {
                        gld<V>(zn, a.zu_next + oc);
                        gld_plain<V>(gv, a.gacc + oc);
                    } else {
#pragma unroll
                        for (int i = 0; i < V; ++i) {
                            zn[i] = P.x0 + i < P.nx ? __ldg(a.zu_next + oc + i) : 0.0f;
                            gv[i] = P.x0 + i < P.nx ? a.gacc[oc + i] : 0.0f;
                        }
                    }
#pragma unroll
                    for (int p = 0; p < V / 2; ++p) {
                        const float2 t = __ffma2_rn(f2(zn[2 * p], zn[2 * p + 1]), f2(d[2 * p], d[2 * p + 1]),
                                                    f2(gv[2 * p], gv[2 * p + 1]));
                        r[2 * p] = t.x;
                        r[2 * p + 1] = t.y;
                    }
                    vput<V>(a.gacc, o, r, P.full, P.x0, P.nx);
                }
            }
        }
        s0.stage(smn, P.tx, P.ty, hm);
        if (NF == 2) s1.stage(smn + G::TILE, P.tx, P.ty, hm);
        s0.shift();
        if (NF == 2) s1.shift();
    }
}

// ------------------------------------------------------------- pass 2, forward
template <int K, int V, int TX, int TY, int CK>
__global__ void __launch_bounds__(TX * TY) ot4v_fwd_kernel(const Ot4FwdArgs A)
{
    using G = G3<K, V, TX, TY>;
    extern __shared__ __align__(16) float smem4[];
    const FwdArgs& a = A.f;
    const Pos3 P = pos3<V, TX, TY, G::BXP>(a.g);
    const int z0 = blockIdx.z * a.zlen;
    if (z0 >= P.nz) return;
    const int z1 = min(z0 + a.zlen, P.nz);
    float ecol[V];
#pragma unroll
    for (int i = 0; i < V; ++i)
        ecol[i] = (P.rowact && P.x0 + i < P.nx) ? __fadd_rn(a.eta[P.nz + P.y], a.eta[P.nz + P.ny + P.x0 + i]) : 0.0f;
    Inj3<V> ij;
    ij.init(a.src, P.y, P.x0, P.nx, P.rowact);
    HaloMap<K, V, TX, TY> hm;
    hm.init(P.tx, P.ty, P.xb, P.x0, P.y, P.nx, P.ny, P.px);
    const float* __restrict__ U = a.u + P.col;
    const float* __restrict__ UP = a.up + P.col;
    const float* __restrict__ W = a.w + P.col;
    VStage<K, V, TX, TY, float> sz;
    sz.start(A.z, P.col, z0, P.pxy, P.cload, hm, smem4, P.tx, P.ty);
    float nu[V], nup[V], nw[V];
    if (P.cload) {
        gld<V>(nu, U + z0 * P.pxy);
        gld<V>(nup, UP + z0 * P.pxy);
        gld<V>(nw, W + z0 * P.pxy);
    } else {
        vzero<V>(nu);
        vzero<V>(nup);
        vzero<V>(nw);
    }
    const int zqmax = P.nz + K - 1;
    for (int z = z0; z < z1; ++z) {
        float* sm = smem4 + ((z - z0) & 1) * G::TILE;
        float* smn = smem4 + (((z - z0) & 1) ^ 1) * G::TILE;
        sz.take();
        float uv[V], upv[V], wv[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            uv[i] = nu[i];
            upv[i] = nup[i];
            wv[i] = nw[i];
        }
        const int zn = min(z + 1, z1 - 1) * P.pxy, zq = min(z + K + 1, zqmax) * P.pxy;
        sz.fetch(A.z, P.col, zq, zn, P.cload, hm);
        if (P.cload) {
            gld<V>(nu, U + zn);
            gld<V>(nup, UP + zn);
            gld<V>(nw, W + zn);
        }
        __syncthreads();
        if (P.cload) {
            float s[V], v[V];
            lap3<K, V, TX, TY>(s, sz.q, sm, P.tx, P.ty, A.c12);
            ij.add(s, a.src, z);
            const float ez = a.eta[z];
            const float* zc = sz.q[K];
#pragma unroll
            for (int p = 0; p < V / 2; ++p) {
                const int i = 2 * p;
                const float2 eta = __fadd2_rn(f2(ez, ez), f2(ecol[i], ecol[i + 1]));
                const float2 r = leap4v(f2(uv[i], uv[i + 1]), f2(upv[i], upv[i + 1]), f2(wv[i], wv[i + 1]),
                                        f2(zc[i], zc[i + 1]), f2(s[i], s[i + 1]), eta, a.hdt);
                v[i] = r.x;
                v[i + 1] = r.y;
            }
            const long long o = (long long)z * P.pxy + P.col;
            vput<V>(a.out, o, v, P.full, P.x0, P.nx);
            if (CK == CK_FP32) {
                vput<V>(static_cast<float*>(a.ck_up), o, uv, P.full, P.x0, P.nx);
            } else if (CK == CK_BF16) {
                st16<__nv_bfloat16, V>(a.ck_u, o, v, P.full, P.x0, P.nx);
                st16<__nv_bfloat16, V>(a.ck_up, o, uv, P.full, P.x0, P.nx);
            } else if (CK == CK_FP16) {
                const bool inf = st16<__half, V>(a.ck_u, o, v, P.full, P.x0, P.nx) |
                                 st16<__half, V>(a.ck_up, o, uv, P.full, P.x0, P.nx);
                if (inf) atomicOr(a.err, 1);
            }
        }
        sz.stage(smn, P.tx, P.ty, hm);
        sz.shift();
    }
}

// ------------------------------------------------------------- pass 3, reverse
template <int K, int V, int TX, int TY, class UT>
__global__ void __launch_bounds__(TX * TY) ot4v_grad_kernel(const Ot4GradArgs a)
{
    using G = G3<K, V, TX, TY>;
    extern __shared__ __align__(16) float smem4[];
    const Pos3 P = pos3<V, TX, TY, G::BXP>(a.g);
    const int z0 = blockIdx.z * a.zlen;
    if (z0 >= P.nz) return;
    const int z1 = min(z0 + a.zlen, P.nz);
    Inj3<V> is;
    is.init(a.src, P.y, P.x0, P.nx, P.rowact);
    HaloMap<K, V, TX, TY> hm;
    hm.init(P.tx, P.ty, P.xb, P.x0, P.y, P.nx, P.ny, P.px);
    const UT* uu = static_cast<const UT*>(a.u);
    const float* __restrict__ L0 = a.l0 + P.col;
    const float* __restrict__ GA = a.gacc + P.col;
    VStage<K, V, TX, TY, UT> su;
    VStage<K, V, TX, TY, float> szu;
    su.start(uu, P.col, z0, P.pxy, P.cload, hm, smem4, P.tx, P.ty);
    szu.start(a.zu, P.col, z0, P.pxy, P.cload, hm, smem4 + G::TILE, P.tx, P.ty);
    float nl[V], ng[V];
    if (P.cload) {
        gld<V>(nl, L0 + z0 * P.pxy);
        gld_plain<V>(ng, GA + z0 * P.pxy);
    } else {
        vzero<V>(nl);
        vzero<V>(ng);
    }
    const int zqmax = P.nz + K - 1;
    for (int z = z0; z < z1; ++z) {
        float* sm = smem4 + ((z - z0) & 1) * (2 * G::TILE);
        float* smn = smem4 + (((z - z0) & 1) ^ 1) * (2 * G::TILE);
        su.take();
        szu.take();
        float lv[V], gv[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            lv[i] = nl[i];
            gv[i] = ng[i];
        }
        const int zn = min(z + 1, z1 - 1) * P.pxy, zq = min(z + K + 1, zqmax) * P.pxy;
        su.fetch(uu, P.col, zq, zn, P.cload, hm);
        szu.fetch(a.zu, P.col, zq, zn, P.cload, hm);
        if (P.cload) {
            gld<V>(nl, L0 + zn);
            gld_plain<V>(ng, GA + zn);
        }
        __syncthreads();
        if (P.cload) {
            float g[V], t[V], acc[V];
            lap3<K, V, TX, TY>(g, su.q, sm, P.tx, P.ty, a.c);
            lap3<K, V, TX, TY>(t, szu.q, sm + G::TILE, P.tx, P.ty, a.c12);
#pragma unroll
            for (int p = 0; p < V / 2; ++p) {
                const float2 r = __fadd2_rn(f2(g[2 * p], g[2 * p + 1]), f2(t[2 * p], t[2 * p + 1]));
                g[2 * p] = r.x;
                g[2 * p + 1] = r.y;
            }
            is.add(g, a.src, z);
#pragma unroll
            for (int p = 0; p < V / 2; ++p) {
                const float2 r = __ffma2_rn(f2(lv[2 * p], lv[2 * p + 1]), f2(g[2 * p], g[2 * p + 1]),
                                            f2(gv[2 * p], gv[2 * p + 1]));
                acc[2 * p] = r.x;
                acc[2 * p + 1] = r.y;
            }
            vput<V>(a.gacc, (long long)z * P.pxy + P.col, acc, P.full, P.x0, P.nx);
        }
        su.stage(smn, P.tx, P.ty, hm);
        szu.stage(smn + G::TILE, P.tx, P.ty, hm);
        su.shift();
        szu.shift();
    }
}

// ---------------------------------------------------------------- dispatch
// (V, TX, TY) shapes: {4, 8, 16} and {2, 16, 16} for every pass.
template <int V, int TX, int TY, int BXP>
dim3 grid4(const FieldGeom& g, int zlen)
{
    return dim3((g.nx + BXP - 1) / BXP, (g.ny + TY - 1) / TY, (g.nz + zlen - 1) / zlen);
}

template <int K, int V, int TX, int TY>
cudaError_t lapv_go(const Ot4LapArgs& a, int ut, cudaStream_t s)
{
    using G = G3<K, V, TX, TY>;
    const dim3 blk(TX, TY, 1), grd = grid4<V, TX, TY, G::BXP>(a.g, a.zlen);
    const int nf = a.f1 ? 2 : 1;
    const size_t sh = 2 * (size_t)nf * G::TILE * sizeof(float);
    if (nf == 1) {
        ot4v_lap_kernel<K, V, TX, TY, 1, float><<<grd, blk, sh, s>>>(a);
    } else {
        switch (ut) {
        case U_FP32: ot4v_lap_kernel<K, V, TX, TY, 2, float><<<grd, blk, sh, s>>>(a); break;
        case U_BF16: ot4v_lap_kernel<K, V, TX, TY, 2, __nv_bfloat16><<<grd, blk, sh, s>>>(a); break;
        case U_FP16: ot4v_lap_kernel<K, V, TX, TY, 2, __half><<<grd, blk, sh, s>>>(a); break;
        default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

template <int K, int V, int TX, int TY>
cudaError_t fwdv_go(const Ot4FwdArgs& a, int ck, cudaStream_t s)
{
    using G = G3<K, V, TX, TY>;
    const dim3 blk(TX, TY, 1), grd = grid4<V, TX, TY, G::BXP>(a.f.g, a.f.zlen);
    const size_t sh = 2 * (size_t)G::TILE * sizeof(float);
    switch (ck) {
    case CK_NONE: ot4v_fwd_kernel<K, V, TX, TY, CK_NONE><<<grd, blk, sh, s>>>(a); break;
    case CK_FP32: ot4v_fwd_kernel<K, V, TX, TY, CK_FP32><<<grd, blk, sh, s>>>(a); break;
    case CK_BF16: ot4v_fwd_kernel<K, V, TX, TY, CK_BF16><<<grd, blk, sh, s>>>(a); break;
    case CK_FP16: ot4v_fwd_kernel<K, V, TX, TY, CK_FP16><<<grd, blk, sh, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int K, int V, int TX, int TY>
cudaError_t gradv_go(const Ot4GradArgs& a, int ut, cudaStream_t s)
{
    using G = G3<K, V, TX, TY>;
    const dim3 blk(TX, TY, 1), grd = grid4<V, TX, TY, G::BXP>(a.g, a.zlen);
    const size_t sh = 4 * (size_t)G::TILE * sizeof(float);
    switch (ut) {
    case U_FP32: ot4v_grad_kernel<K, V, TX, TY, float><<<grd, blk, sh, s>>>(a); break;
    case U_BF16: ot4v_grad_kernel<K, V, TX, TY, __nv_bfloat16><<<grd, blk, sh, s>>>(a); break;
    case U_FP16: ot4v_grad_kernel<K, V, TX, TY, __half><<<grd, blk, sh, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int K>
cudaError_t gradv_k(const Ot4GradArgs& a, const Tile& t, int ut, cudaStream_t s)
{
    if (t.vec == 4) return gradv_go<K, 4, 8, 16>(a, ut, s);
    return gradv_go<K, 2, 16, 16>(a, ut, s);
}

template <int K>
cudaError_t lapv_k(const Ot4LapArgs& a, const Tile& t, int ut, cudaStream_t s)
{
    if (t.vec == 4) return lapv_go<K, 4, 8, 16>(a, ut, s);
    return lapv_go<K, 2, 16, 16>(a, ut, s);
}

template <int K>
cudaError_t fwdv_k(const Ot4FwdArgs& a, const Tile& t, int ck, cudaStream_t s)
{
    if (t.vec == 4) return fwdv_go<K, 4, 8, 16>(a, ck, s);
    return fwdv_go<K, 2, 16, 16>(a, ck, s);
}
}  // namespace

bool ot4v_supported(int dims, int K, const Tile& t, bool reverse)
{
    (void)reverse;   // every pass has both vector widths
    if (dims != 3 || t.ver != 6 || t.zlen < 1 || t.by != 16 || t.bx != 32 || t.by < K) return false;
    if (K != 1 && K != 2 && K != 4 && K != 8) return false;
    return t.vec == 2 || t.vec == 4;
}

cudaError_t launch_ot4v_lap(const Ot4LapArgs& a, const Tile& t, int K, int ut, cudaStream_t s)
{
    Ot4LapArgs b = a;
    b.zlen = t.zlen;
    if (!v3_fits(a.g, K) || !ot4v_supported(a.g.dims, K, t, a.f1 != nullptr)) return cudaErrorInvalidValue;
    switch (K) {
    case 1: return lapv_k<1>(b, t, ut, s);
    case 2: return lapv_k<2>(b, t, ut, s);
    case 4: return lapv_k<4>(b, t, ut, s);
    case 8: return lapv_k<8>(b, t, ut, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ot4v_fwd(const Ot4FwdArgs& a, const Tile& t, int K, int ck, cudaStream_t s)
{
    Ot4FwdArgs b = a;
    b.f.zlen = t.zlen;
    if (!v3_fits(a.f.g, K) || !ot4v_supported(a.f.g.dims, K, t, false)) return cudaErrorInvalidValue;
    switch (K) {
    case 1: return fwdv_k<1>(b, t, ck, s);
    case 2: return fwdv_k<2>(b, t, ck, s);
    case 4: return fwdv_k<4>(b, t, ck, s);
    case 8: return fwdv_k<8>(b, t, ck, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ot4v_grad(const Ot4GradArgs& a, const Tile& t, int K, int ut, cudaStream_t s)
{
    Ot4GradArgs b = a;
    b.zlen = t.zlen;
    if (!v3_fits(a.g, K) || !ot4v_supported(a.g.dims, K, t, true)) return cudaErrorInvalidValue;
    switch (K) {
    case 1: return gradv_k<1>(b, t, ut, s);
    case 2: return gradv_k<2>(b, t, ut, s);
    case 4: return gradv_k<4>(b, t, ut, s);
    case 8: return gradv_k<8>(b, t, ut, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ckfwi
