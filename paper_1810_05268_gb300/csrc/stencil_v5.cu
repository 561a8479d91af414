// Lean forward and fused reverse OT2 steps fed by asynchronous copies (3D,
// Tile.ver 7).
//
// The async-copy kernels (stencil_v4.cu) issue about 360 instructions per
// warp and plane at order 8, of which about 130 are the stencil's
// floating-point operations and 22 memory instructions: the rest is integer
// and control work (copy addresses and their predicates rebuilt every plane,
// ring indices, packed-operand pairs).  The steps are issue-bound, so this
// generation keeps their arithmetic -- the same operations in the same order
// (lap3's difference-form Laplacian, leap2v's increment-form update), so the
// results are bitwise those of every other generation -- and strips the
// bookkeeping:
//   * every copy of a thread (its u-tile vector, its halo vectors, its point
//     vectors) is described once, before the plane loop, by a shared-memory
//     offset, an element offset from the plane origin and a byte count
//     (16, or 0 for a zero-filled copy whose source is never read); a plane
//     then costs one address add per copy;
//   * the plane index of a prefetch is clamped to the last valid plane
//     instead of predicating the copy;
//   * the stencil coefficients and the update's constants are packed into
//     register pairs once;
//   * NP = 2 computes two planes per iteration: one barrier, one wait and
//     one queue shift (by two) for every two planes, and two planes of
//     independent work between them.
// Step (NP planes z .. z+NP-1): wait for the previous group of copies (u
// tiles z+K .. z+K+NP-1 and point planes z .. z+NP-1), barrier, issue the
// next group (u tiles z+K+NP .. z+K+2NP-1, point planes z+NP .. z+2NP-1)
// into the slots of the planes computed in the previous step, compute.
#include "stencil_v3.cuh"

namespace ckfwi {
namespace {

constexpr int V5 = 4;
constexpr int TX5 = 8;
constexpr int TY5 = 16;

template <int K, int NP>
struct G5 {
    using G = G3<K, V5, TX5, TY5>;
    static constexpr int RU = K + 2 * NP;               // u tiles in flight
    static constexpr int RP = 2 * NP;                   // planes of each point ring
    static constexpr int PT = G::BXP * TY5;             // floats of a point tile
    static constexpr int NT = TX5 * TY5;                // threads
    static constexpr int NXH = 2 * TY5 * (G::PX / V5);  // x-halo vectors of a u tile
    static constexpr int NYH = 2 * K * (G::BXP / V5);   // y-halo vectors
    static constexpr int NH = NXH + NYH;
    static constexpr int HPT = (NH + NT - 1) / NT;      // halo vectors per thread
    static constexpr unsigned TB = G::TILE * 4u;        // bytes of a u tile
    static constexpr unsigned PB = PT * 4u;             // bytes of a point tile
};

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// 16 bytes global -> shared, asynchronously; n = 0 zero-fills (nothing is read)
__device__ __forceinline__ void cp16(unsigned dst, const float* src, unsigned n)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_commit5() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait5_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// One thread's copies of a plane, described once: shared-memory byte offset
// inside a tile, element offset from the plane's origin, and byte count (an
// invalid copy reads nothing and points at the plane origin).
template <int K, int NP>
struct Desc5 {
    using H = G5<K, NP>;
    using G = typename H::G;
    unsigned cd, cn;             // centre vector: offset in a u tile, bytes
    int cs;                      // and element offset (also the point vectors')
    unsigned pd;                 // offset of the thread's vector in a point tile
    unsigned hd[H::HPT], hn[H::HPT];
    int hs[H::HPT];
    bool hon[H::HPT];            // the thread has this halo vector at all
    __device__ __forceinline__ void init(int tid, int tx, int ty, int xb, int yb, int nx, int ny, int px)
    {
        const int x0 = xb + V5 * tx, y = yb + ty;
        const bool cv = y < ny && x0 < nx;
        cd = 4u * (unsigned)((ty + K) * G::RX + G::PX + V5 * tx);
        cs = cv ? y * px + x0 : 0;
        cn = cv ? 16u : 0u;
        pd = 4u * (unsigned)(ty * G::BXP + V5 * tx);
#pragma unroll
        for (int k = 0; k < H::HPT; ++k) {
            const int h = tid + k * H::NT;
            bool v = false;
            int off = 0, so = 0;
            hon[k] = h < H::NH;
            if (h < H::NXH) {
                constexpr int PV = G::PX / V5;                  // vectors per halo row
                const int side = h / (TY5 * PV), rem = h % (TY5 * PV);
                const int r = rem / PV, c = rem % PV;
                const int yy = yb + r;
                const int xx = (side ? xb + G::BXP : xb - G::PX) + c * V5;
                v = yy < ny && (side == 0 || xb + G::BXP < nx + K);
                off = yy * px + xx;
                so = (r + K) * G::RX + (side ? G::PX + G::BXP : 0) + c * V5;
            } else if (h < H::NH) {
                constexpr int BV = G::BXP / V5;                 // vectors per halo row
                const int h2 = h - H::NXH;
                const int side = h2 / (K * BV), rem = h2 % (K * BV);
                const int rr = rem / BV, c = rem % BV;
                const int yy = side ? yb + TY5 + rr : yb - K + rr;
                const int xx = xb + c * V5;
                v = xx < nx && (side == 0 || yy < ny + K);
                off = yy * px + xx;
                so = (side ? TY5 + K + rr : rr) * G::RX + G::PX + c * V5;
            }
            hd[k] = 4u * (unsigned)so;
            hs[k] = v ? off : 0;
            hn[k] = v ? 16u : 0u;
        }
    }
    // the halo'd u tile of the plane whose origin is `pl`, into the tile at `slot`
    __device__ __forceinline__ void tile(unsigned slot, const float* pl) const
    {
        cp16(slot + cd, pl + cs, cn);
#pragma unroll
        for (int k = 0; k < H::HPT; ++k)
            if (hon[k]) cp16(slot + hd[k], pl + hs[k], hn[k]);
    }
    __device__ __forceinline__ void point(unsigned slot, const float* pl) const { cp16(slot + pd, pl + cs, cn); }
};

// lap3's Laplacian with the queue window starting at q[M] (compile-time) and
// the coefficient pairs precomputed: the same operations in the same order.
template <int K, int M, int NQ>
__device__ __forceinline__ void lap5(float (&out)[V5], const float (&q)[NQ][V5], const float* sm, int tx, int ty,
                                     const float2 (&cj2)[K + 1])
{
    using G = G3<K, V5, TX5, TY5>;
    const int r = ty + K;
    float xw[V5 + 2 * G::PX];
#pragma unroll
    for (int k = 0; k < G::NW; ++k) {
        float t[V5];
        sld<V5>(t, sm + r * G::RX + V5 * tx + V5 * k);
#pragma unroll
        for (int i = 0; i < V5; ++i) xw[V5 * k + i] = t[i];
    }
    const float* u = q[M + K];
    float2 nu[V5 / 2], acc[V5 / 2];
#pragma unroll
    for (int p = 0; p < V5 / 2; ++p) {
        nu[p] = f2(-u[2 * p], -u[2 * p + 1]);
        acc[p] = f2(0.0f, 0.0f);
    }
#pragma unroll
    for (int j = K; j >= 1; --j) {
        float yp[V5], ym[V5];
        sld<V5>(yp, sm + (r + j) * G::RX + G::PX + V5 * tx);
        sld<V5>(ym, sm + (r - j) * G::RX + G::PX + V5 * tx);
        const float* zp = q[M + K + j];
        const float* zm = q[M + K - j];
#pragma unroll
        for (int p = 0; p < V5 / 2; ++p) {
            const int i = 2 * p;
            float2 s = __fadd2_rn(__fadd2_rn(f2(zp[i], zp[i + 1]), nu[p]), __fadd2_rn(f2(zm[i], zm[i + 1]), nu[p]));
            float2 sx;
            if (j % 2 == 0) {
                sx = __fadd2_rn(__fadd2_rn(f2(xw[G::PX + i + j], xw[G::PX + i + 1 + j]), nu[p]),
                                __fadd2_rn(f2(xw[G::PX + i - j], xw[G::PX + i + 1 - j]), nu[p]));
            } else {
                sx.x = __fadd_rn(__fsub_rn(xw[G::PX + i + j], u[i]), __fsub_rn(xw[G::PX + i - j], u[i]));
                sx.y = __fadd_rn(__fsub_rn(xw[G::PX + i + 1 + j], u[i + 1]), __fsub_rn(xw[G::PX + i + 1 - j], u[i + 1]));
            }
            s = __fadd2_rn(s, sx);
            const float2 sy = __fadd2_rn(__fadd2_rn(f2(yp[i], yp[i + 1]), nu[p]), __fadd2_rn(f2(ym[i], ym[i + 1]), nu[p]));
            s = __fadd2_rn(s, sy);
            acc[p] = __ffma2_rn(cj2[j], s, acc[p]);
        }
    }
#pragma unroll
    for (int p = 0; p < V5 / 2; ++p) {
        out[2 * p] = acc[p].x;
        out[2 * p + 1] = acc[p].y;
    }
}

// the next slot of a ring of R slots of B bytes starting at `base`
template <int R, unsigned B>
__device__ __forceinline__ unsigned nxt(unsigned s, unsigned base, int n = 1)
{
    s += (unsigned)n * B;
    return s >= base + (unsigned)R * B ? s - (unsigned)R * B : s;
}

// Plane zz of the forward step: stencil on the staged tile at smem `sm`
// (generic pointer), queue window q[M .. M + 2K], point values from the
// rings; writes u^{n+1} and the fused checkpoint copies.
template <int K, int M, int NQ, int CK>
__device__ __forceinline__ void fwd5_plane(const FwdArgs& a, const float (&q)[NQ][V5], const float* sm,
                                           const float* upt, const float* wpt, int zz, int tx, int ty,
                                           const float2 (&cj2)[K + 1], const float (&ecol)[V5], const Inj3<V5>& ij,
                                           float* __restrict__ OUT, long long col, long long pxy, bool full, int x0,
                                           int nx)
{
    float upv[V5], wv[V5];
    sld<V5>(upv, upt);
    sld<V5>(wv, wpt);
    const float* uc = q[M + K];
    float s[V5];
    lap5<K, M, NQ>(s, q, sm, tx, ty, cj2);
    ij.add(s, a.src, zz);
    const float ez = a.eta[zz];
    float v[V5];
#pragma unroll
    for (int p = 0; p < V5 / 2; ++p) {
        const int i = 2 * p;
        const float2 eta = __fadd2_rn(f2(ez, ez), f2(ecol[i], ecol[i + 1]));
        const float2 r = leap2v(f2(uc[i], uc[i + 1]), f2(upv[i], upv[i + 1]), f2(wv[i], wv[i + 1]),
                                f2(s[i], s[i + 1]), eta, a.hdt);
        v[i] = r.x;
        v[i + 1] = r.y;
    }
    const long long o = (long long)zz * pxy + col;
    if (full) {
        vst<V5>(OUT + o, v);
        if (CK == CK_FP32) vstp<V5>(static_cast<float*>(a.ck_up) + o, uc);
    } else {
#pragma unroll
        for (int i = 0; i < V5; ++i) {
            if (x0 + i < nx) {
                OUT[o + i] = v[i];
                if (CK == CK_FP32) static_cast<float*>(a.ck_up)[o + i] = uc[i];
            }
        }
    }
    if (CK == CK_BF16) {
        st16<__nv_bfloat16, V5>(a.ck_u, o, v, full, x0, nx);
        st16<__nv_bfloat16, V5>(a.ck_up, o, uc, full, x0, nx);
    } else if (CK == CK_FP16) {
        const bool inf = st16<__half, V5>(a.ck_u, o, v, full, x0, nx) | st16<__half, V5>(a.ck_up, o, uc, full, x0, nx);
        if (inf) atomicOr(a.err, 1);
    }
}

template <int K, int NP, int CK>
__device__ __forceinline__ void fwd5_body(const FwdArgs& a, float* smem, int bxi, int byi, int bzi, int gxn, int gyn)
{
    using H = G5<K, NP>;
    using G = typename H::G;
    constexpr int NQ = 2 * K + NP;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX5 + tx;
    const int nz = a.g.nz, ny = a.g.ny, nx = a.g.nx;
    const int px = (int)a.g.px;
    const long long pxy = a.g.pxy;
    const int xb = bxi * G::BXP, yb = byi * TY5;
    const int x0 = xb + V5 * tx;
    const int y = yb + ty;

    if (a.smp.n > 0) {   // receiver sampling of u^n by the first threads of the grid
        const int gt = ((bzi * gyn + byi) * gxn + bxi) * H::NT + tid;
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
    const bool rowact = y < ny;
    const bool cload = rowact && x0 < nx;
    const bool full = rowact && x0 + V5 <= nx;
    const long long col = (long long)y * px + x0;
    float ecol[V5];
#pragma unroll
    for (int i = 0; i < V5; ++i)
        ecol[i] = (rowact && x0 + i < nx) ? __fadd_rn(a.eta[nz + y], a.eta[nz + ny + x0 + i]) : 0.0f;
    float2 cj2[K + 1];
#pragma unroll
    for (int j = 0; j <= K; ++j) cj2[j] = f2(a.c[j], a.c[j]);
    Inj3<V5> ij;
    ij.init(a.src, y, x0, nx, rowact);
    Desc5<K, NP> d;
    d.init(tid, tx, ty, xb, yb, nx, ny, px);

    const unsigned ub = su32(smem);                         // RU u tiles
    const unsigned pb = ub + H::RU * H::TB;                 // RP point tiles of u^{n-1}
    const unsigned wb = pb + H::RP * H::PB;                 // RP point tiles of w
    const float* ringf = smem;
    const int zumax = nz + K - 1;                           // last plane with memory (zero halo)

    float q[NQ][V5];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        if (cload) gld<V5>(q[i], a.u + (long long)(z0 - K + i) * pxy + col);
        else vzero<V5>(q[i]);
    }
    // prologue: u tiles z0 .. z0 + K + NP - 1, point planes z0 .. z0 + NP - 1
#pragma unroll 1
    for (int p = 0; p < K + NP; ++p) d.tile(ub + p * H::TB, a.u + (long long)min(z0 + p, zumax) * pxy);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const long long po = (long long)min(z0 + p, z1 - 1) * pxy;
        d.point(pb + p * H::PB, a.up + po);
        d.point(wb + p * H::PB, a.w + po);
    }
    cp_commit5();
    cp_wait5_all();
    __syncthreads();
#pragma unroll
    for (int i = 0; i < K; ++i) sld<V5>(q[K + i], ringf + i * G::TILE + d.cd / 4);

    unsigned su = ub, sp = pb;       // slots of plane z (u ring) and of point plane z
    for (int z = z0; z < z1; z += NP) {
        if (z > z0) {
            cp_wait5_all();
            __syncthreads();
        }
        // the next group: u tiles z+K+NP .. z+K+2NP-1, point planes z+NP .. z+2NP-1
        {
            unsigned sn = nxt<H::RU, H::TB>(su, ub, K + NP);
            unsigned pn = nxt<H::RP, H::PB>(sp, pb, NP);
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                d.tile(sn, a.u + (long long)min(z + K + NP + m, zumax) * pxy);
                const long long po = (long long)min(z + NP + m, z1 - 1) * pxy;
                d.point(pn, a.up + po);
                d.point(pn + H::RP * H::PB, a.w + po);
                sn = nxt<H::RU, H::TB>(sn, ub);
                pn = nxt<H::RP, H::PB>(pn, pb);
            }
            cp_commit5();
        }
        // the queue's new planes z+K .. z+K+NP-1 from their tiles
        {
            unsigned sk = nxt<H::RU, H::TB>(su, ub, K);
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                sld<V5>(q[2 * K + m], ringf + (sk - ub + d.cd) / 4);
                sk = nxt<H::RU, H::TB>(sk, ub);
            }
        }
        if (cload) {
            fwd5_plane<K, 0, NQ, CK>(a, q, ringf + (su - ub) / 4, ringf + (sp - ub + d.pd) / 4,
                                     ringf + (sp + H::RP * H::PB - ub + d.pd) / 4, z, tx, ty, cj2, ecol, ij, a.out,
                                     col, pxy, full, x0, nx);
            if (NP == 2 && z + 1 < z1) {
                const unsigned su1 = nxt<H::RU, H::TB>(su, ub), sp1 = nxt<H::RP, H::PB>(sp, pb);
                fwd5_plane<K, NP - 1, NQ, CK>(a, q, ringf + (su1 - ub) / 4, ringf + (sp1 - ub + d.pd) / 4,
                                              ringf + (sp1 + H::RP * H::PB - ub + d.pd) / 4, z + 1, tx, ty, cj2,
                                              ecol, ij, a.out, col, pxy, full, x0, nx);
            }
        }
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) {
#pragma unroll
            for (int k = 0; k < V5; ++k) q[i][k] = q[i + NP][k];
        }
        su = nxt<H::RU, H::TB>(su, ub, NP);
        sp = nxt<H::RP, H::PB>(sp, pb, NP);
    }
    cp_wait5_all();     // no copy may land after the CTA has left
}

// occupancy: NP = 1 at order <= 8 holds 31 KB of shared memory a CTA, six
// CTAs an SM at <= 80 registers
template <int K, int NP>
constexpr int fwd5_min_blocks() { return NP == 1 && K <= 4 ? 6 : (K <= 4 ? 4 : 1); }

template <int K, int NP, int CK>
__global__ void __launch_bounds__(TX5 * TY5, fwd5_min_blocks<K, NP>()) fwd5_kernel(const FwdArgs a)
{
    extern __shared__ __align__(16) float smem5[];
    fwd5_body<K, NP, CK>(a, smem5, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y);
}

template <int K, int NP>
constexpr size_t fwd5_smem() { return ((size_t)G5<K, NP>::RU * G5<K, NP>::TB) + 2 * (size_t)G5<K, NP>::RP * G5<K, NP>::PB; }

template <int K, int NP>
cudaError_t fwd5_go(const FwdArgs& a, int ck, cudaStream_t s)
{
    using G = typename G5<K, NP>::G;
    const dim3 blk(TX5, TY5, 1);
    const dim3 grd((a.g.nx + G::BXP - 1) / G::BXP, (a.g.ny + TY5 - 1) / TY5, (a.g.nz + a.zlen - 1) / a.zlen);
    const size_t sh = fwd5_smem<K, NP>();
    cudaError_t e = cudaSuccess;
    switch (ck) {
    case CK_NONE:
        e = cudaFuncSetAttribute(fwd5_kernel<K, NP, CK_NONE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        if (e == cudaSuccess) fwd5_kernel<K, NP, CK_NONE><<<grd, blk, sh, s>>>(a);
        break;
    case CK_FP32:
        e = cudaFuncSetAttribute(fwd5_kernel<K, NP, CK_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        if (e == cudaSuccess) fwd5_kernel<K, NP, CK_FP32><<<grd, blk, sh, s>>>(a);
        break;
    case CK_BF16:
        e = cudaFuncSetAttribute(fwd5_kernel<K, NP, CK_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        if (e == cudaSuccess) fwd5_kernel<K, NP, CK_BF16><<<grd, blk, sh, s>>>(a);
        break;
    case CK_FP16:
        e = cudaFuncSetAttribute(fwd5_kernel<K, NP, CK_FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        if (e == cudaSuccess) fwd5_kernel<K, NP, CK_FP16><<<grd, blk, sh, s>>>(a);
        break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int K>
cudaError_t fwd5_k(const FwdArgs& a, const Tile& t, int ck, cudaStream_t s)
{
    if (t.pf == 2) return fwd5_go<K, 2>(a, ck, s);
    return fwd5_go<K, 1>(a, ck, s);
}

// ------------------------------------------------------------- reverse
// Plane zz of the fused reverse step: the adjoint update from the staged
// lam^j tile and queue, the Laplacian of u^{j-1} from its tile and queue,
// the imaging condition into gacc (adj3's operations in its order).
template <int K, int M, int NQ>
__device__ __forceinline__ void adj5_plane(const AdjArgs& a, const float (&ql)[NQ][V5], const float (&qu)[NQ][V5],
                                           const float* sl, const float* su_, const float* l2t, const float* wt,
                                           const float* gt, int zz, int tx, int ty, const float2 (&cj2)[K + 1],
                                           const float (&ecol)[V5], const Inj3<V5>& ia, const Inj3<V5>& is,
                                           long long col, long long pxy, bool full, int x0, int nx)
{
    float l2v[V5], wv[V5], gv[V5];
    sld<V5>(l2v, l2t);
    sld<V5>(wv, wt);
    sld<V5>(gv, gt);
    float sl_[V5], su2[V5];
    lap5<K, M, NQ>(sl_, ql, sl, tx, ty, cj2);
    ia.add(sl_, a.adj, zz);
    lap5<K, M, NQ>(su2, qu, su_, tx, ty, cj2);
    is.add(su2, a.src, zz);
    const float* lc = ql[M + K];
    const float ez = a.eta[zz];
    float lam[V5], gn[V5];
#pragma unroll
    for (int p = 0; p < V5 / 2; ++p) {
        const int i = 2 * p;
        const float2 eta = __fadd2_rn(f2(ez, ez), f2(ecol[i], ecol[i + 1]));
        const float2 r = leap2v(f2(lc[i], lc[i + 1]), f2(l2v[i], l2v[i + 1]), f2(wv[i], wv[i + 1]),
                                f2(sl_[i], sl_[i + 1]), eta, a.hdt);
        const float2 gg = __ffma2_rn(r, f2(su2[i], su2[i + 1]), f2(gv[i], gv[i + 1]));
        lam[i] = r.x;
        lam[i + 1] = r.y;
        gn[i] = gg.x;
        gn[i + 1] = gg.y;
    }
    const long long o = (long long)zz * pxy + col;
    if (full) {
        vst<V5>(a.l0 + o, lam);
        vst<V5>(a.gacc + o, gn);
    } else {
#pragma unroll
        for (int i = 0; i < V5; ++i) {
            if (x0 + i < nx) {
                a.l0[o + i] = lam[i];
                a.gacc[o + i] = gn[i];
            }
        }
    }
}

template <int K, int NP>
__device__ __forceinline__ void adj5_body(const AdjArgs& a, float* smem, int bxi, int byi, int bzi)
{
    using H = G5<K, NP>;
    using G = typename H::G;
    constexpr int NQ = 2 * K + NP;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX5 + tx;
    const int nz = a.g.nz, ny = a.g.ny, nx = a.g.nx;
    const int px = (int)a.g.px;
    const long long pxy = a.g.pxy;
    const int xb = bxi * G::BXP, yb = byi * TY5;
    const int x0 = xb + V5 * tx;
    const int y = yb + ty;
    const int z0 = bzi * a.zlen;
    if (z0 >= nz) return;
    const int z1 = min(z0 + a.zlen, nz);
    const bool rowact = y < ny;
    const bool cload = rowact && x0 < nx;
    const bool full = rowact && x0 + V5 <= nx;
    const long long col = (long long)y * px + x0;
    float ecol[V5];
#pragma unroll
    for (int i = 0; i < V5; ++i)
        ecol[i] = (rowact && x0 + i < nx) ? __fadd_rn(a.eta[nz + y], a.eta[nz + ny + x0 + i]) : 0.0f;
    float2 cj2[K + 1];
#pragma unroll
    for (int j = 0; j <= K; ++j) cj2[j] = f2(a.c[j], a.c[j]);
    Inj3<V5> ia, is;
    ia.init(a.adj, y, x0, nx, rowact);
    is.init(a.src, y, x0, nx, rowact);
    Desc5<K, NP> d;
    d.init(tid, tx, ty, xb, yb, nx, ny, px);
    const float* uu = static_cast<const float*>(a.u);

    constexpr unsigned FR = H::RU * H::TB;                  // bytes of one u-tile ring
    constexpr unsigned PR = H::RP * H::PB;                  // bytes of one point ring
    const unsigned lb = su32(smem);                         // lam^j tiles, then u^{j-1} tiles (+FR)
    const unsigned pb = lb + 2 * FR;                        // lam^{j+1}, w (+PR), gacc (+2PR) point rings
    const float* ringf = smem;
    const int zumax = nz + K - 1;

    float ql[NQ][V5], qu[NQ][V5];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const long long o = (long long)(z0 - K + i) * pxy + col;
        if (cload) {
            gld<V5>(ql[i], a.l1 + o);
            gld<V5>(qu[i], uu + o);
        } else {
            vzero<V5>(ql[i]);
            vzero<V5>(qu[i]);
        }
    }
#pragma unroll 1
    for (int p = 0; p < K + NP; ++p) {
        const long long o = (long long)min(z0 + p, zumax) * pxy;
        d.tile(lb + p * H::TB, a.l1 + o);
        d.tile(lb + FR + p * H::TB, uu + o);
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const long long po = (long long)min(z0 + p, z1 - 1) * pxy;
        d.point(pb + p * H::PB, a.l2 + po);
        d.point(pb + PR + p * H::PB, a.w + po);
        d.point(pb + 2 * PR + p * H::PB, a.gacc + po);
    }
    cp_commit5();
    cp_wait5_all();
    __syncthreads();
#pragma unroll
    for (int i = 0; i < K; ++i) {
        sld<V5>(ql[K + i], ringf + i * G::TILE + d.cd / 4);
        sld<V5>(qu[K + i], ringf + (FR / 4) + i * G::TILE + d.cd / 4);
    }

    unsigned sl = lb, sp = pb;
    for (int z = z0; z < z1; z += NP) {
        if (z > z0) {
            cp_wait5_all();
            __syncthreads();
        }
        {
            unsigned sn = nxt<H::RU, H::TB>(sl, lb, K + NP);
            unsigned pn = nxt<H::RP, H::PB>(sp, pb, NP);
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                const long long o = (long long)min(z + K + NP + m, zumax) * pxy;
                d.tile(sn, a.l1 + o);
                d.tile(sn + FR, uu + o);
                const long long po = (long long)min(z + NP + m, z1 - 1) * pxy;
                d.point(pn, a.l2 + po);
                d.point(pn + PR, a.w + po);
                d.point(pn + 2 * PR, a.gacc + po);
                sn = nxt<H::RU, H::TB>(sn, lb);
                pn = nxt<H::RP, H::PB>(pn, pb);
            }
            cp_commit5();
        }
        {
            unsigned sk = nxt<H::RU, H::TB>(sl, lb, K);
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                sld<V5>(ql[2 * K + m], ringf + (sk - lb + d.cd) / 4);
                sld<V5>(qu[2 * K + m], ringf + (sk + FR - lb + d.cd) / 4);
                sk = nxt<H::RU, H::TB>(sk, lb);
            }
        }
        if (cload) {
            const float* t0 = ringf + (sl - lb) / 4;
            const float* p0 = ringf + (sp - lb + d.pd) / 4;
            adj5_plane<K, 0, NQ>(a, ql, qu, t0, t0 + FR / 4, p0, p0 + PR / 4, p0 + 2 * PR / 4, z, tx, ty, cj2, ecol,
                                 ia, is, col, pxy, full, x0, nx);
            if (NP == 2 && z + 1 < z1) {
                const float* t1 = ringf + (nxt<H::RU, H::TB>(sl, lb) - lb) / 4;
                const float* p1 = ringf + (nxt<H::RP, H::PB>(sp, pb) - lb + d.pd) / 4;
                adj5_plane<K, NP - 1, NQ>(a, ql, qu, t1, t1 + FR / 4, p1, p1 + PR / 4, p1 + 2 * PR / 4, z + 1, tx,
                                          ty, cj2, ecol, ia, is, col, pxy, full, x0, nx);
            }
        }
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) {
#pragma unroll
            for (int k = 0; k < V5; ++k) {
                ql[i][k] = ql[i + NP][k];
                qu[i][k] = qu[i + NP][k];
            }
        }
        sl = nxt<H::RU, H::TB>(sl, lb, NP);
        sp = nxt<H::RP, H::PB>(sp, pb, NP);
    }
    cp_wait5_all();
}

// NP = 1 at order <= 8: 58 KB of shared memory a CTA, three CTAs an SM at
// <= 168 registers
template <int K, int NP>
constexpr int adj5_min_blocks() { return NP == 1 && K <= 4 ? 3 : 1; }

template <int K, int NP>
__global__ void __launch_bounds__(TX5 * TY5, adj5_min_blocks<K, NP>()) adj5_kernel(const AdjArgs a)
{
    extern __shared__ __align__(16) float smem5[];
    adj5_body<K, NP>(a, smem5, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <int K, int NP>
constexpr size_t adj5_smem() { return 2 * ((size_t)G5<K, NP>::RU * G5<K, NP>::TB) + 3 * (size_t)G5<K, NP>::RP * G5<K, NP>::PB; }

template <int K, int NP>
cudaError_t adj5_go(const AdjArgs& a, cudaStream_t s)
{
    using G = typename G5<K, NP>::G;
    const dim3 blk(TX5, TY5, 1);
    const dim3 grd((a.g.nx + G::BXP - 1) / G::BXP, (a.g.ny + TY5 - 1) / TY5, (a.g.nz + a.zlen - 1) / a.zlen);
    const size_t sh = adj5_smem<K, NP>();
    cudaError_t e = cudaFuncSetAttribute(adj5_kernel<K, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (e != cudaSuccess) return e;
    adj5_kernel<K, NP><<<grd, blk, sh, s>>>(a);
    return cudaGetLastError();
}

template <int K>
cudaError_t adj5_k(const AdjArgs& a, const Tile& t, cudaStream_t s)
{
    if (t.pf == 2) return adj5_go<K, 2>(a, s);
    return adj5_go<K, 1>(a, s);
}

// ------------------------------------------------------------- batches
// One launch advances every lane of a batch: lane l's CTAs are laid out
// like its own single-lane grid (x fastest, then y, then z runs) and its
// arguments are staged from a device table (the single-lane bodies above,
// so every lane's values are bitwise a single-shot run's).
template <int K, int NP>
__global__ void __launch_bounds__(TX5 * TY5, adj5_min_blocks<K, NP>())
    adj5_batch_kernel(const AdjArgs* __restrict__ tab, const int* __restrict__ start, int nl)
{
    using G = typename G5<K, NP>::G;
    extern __shared__ __align__(16) float smem5[];
    __shared__ __align__(16) AdjArgs a;
    const int b = stage_args(a, tab, start, nl);
    const int gx = (a.g.nx + G::BXP - 1) / G::BXP;
    const int gy = (a.g.ny + TY5 - 1) / TY5;
    adj5_body<K, NP>(a, smem5, b % gx, (b / gx) % gy, b / (gx * gy));
}

template <int K, int NP, int CK>
__global__ void __launch_bounds__(TX5 * TY5, fwd5_min_blocks<K, NP>())
    fwd5_batch_kernel(const FwdArgs* __restrict__ tab, const int* __restrict__ start, int nl)
{
    using G = typename G5<K, NP>::G;
    extern __shared__ __align__(16) float smem5[];
    __shared__ __align__(16) FwdArgs a;
    const int b = stage_args(a, tab, start, nl);
    const int gx = (a.g.nx + G::BXP - 1) / G::BXP;
    const int gy = (a.g.ny + TY5 - 1) / TY5;
    fwd5_body<K, NP, CK>(a, smem5, b % gx, (b / gx) % gy, b / (gx * gy), gx, gy);
}

template <int K, int NP>
cudaError_t adj5b_go(const BatchLaunch<AdjArgs>& b, cudaStream_t s)
{
    const size_t sh = adj5_smem<K, NP>();
    cudaError_t e = cudaFuncSetAttribute(adj5_batch_kernel<K, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sh);
    if (e != cudaSuccess) return e;
    adj5_batch_kernel<K, NP><<<dim3((unsigned)b.blocks), dim3(TX5, TY5), sh, s>>>(b.tab, b.start, b.lanes);
    return cudaGetLastError();
}

template <int K, int NP, int CK>
cudaError_t fwd5b_ck(const BatchLaunch<FwdArgs>& b, cudaStream_t s)
{
    const size_t sh = fwd5_smem<K, NP>();
    cudaError_t e = cudaFuncSetAttribute(fwd5_batch_kernel<K, NP, CK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sh);
    if (e != cudaSuccess) return e;
    fwd5_batch_kernel<K, NP, CK><<<dim3((unsigned)b.blocks), dim3(TX5, TY5), sh, s>>>(b.tab, b.start, b.lanes);
    return cudaGetLastError();
}

template <int K, int NP>
cudaError_t fwd5b_go(const BatchLaunch<FwdArgs>& b, int ck, cudaStream_t s)
{
    switch (ck) {
    case CK_NONE: return fwd5b_ck<K, NP, CK_NONE>(b, s);
    case CK_FP32: return fwd5b_ck<K, NP, CK_FP32>(b, s);
    case CK_BF16: return fwd5b_ck<K, NP, CK_BF16>(b, s);
    case CK_FP16: return fwd5b_ck<K, NP, CK_FP16>(b, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool v5_supported(int dims, int K, const Tile& t)
{
    if (dims != 3 || t.ver != 7 || t.zlen < 1) return false;
    if (K != 1 && K != 2 && K != 4 && K != 8) return false;
    if (t.bx != V5 * TX5 || t.by != TY5 || t.vec != V5 || (t.pf != 1 && t.pf != 2)) return false;
    // shared memory per CTA within the 227 KB an SM offers one CTA
    const size_t sh = t.pf == 2 ? (K == 8 ? adj5_smem<8, 2>() : adj5_smem<4, 2>())
                                : (K == 8 ? adj5_smem<8, 1>() : adj5_smem<4, 1>());
    return sh <= 227u * 1024u;
}

cudaError_t launch_fwd5(const FwdArgs& a, const Tile& t, int K, int ck, cudaStream_t s)
{
    FwdArgs b = a;
    b.zlen = t.zlen;
    if (!v3_fits(a.g, K) || !v5_supported(a.g.dims, K, t)) return cudaErrorInvalidValue;
    switch (K) {
    case 1: return fwd5_k<1>(b, t, ck, s);
    case 2: return fwd5_k<2>(b, t, ck, s);
    case 4: return fwd5_k<4>(b, t, ck, s);
    case 8: return fwd5_k<8>(b, t, ck, s);
    default: return cudaErrorInvalidValue;
    }
}

// FP32 u^{j-1} only; 16-bit checkpoints are up-cast before a reverse step
// (the executor), and the vector-blocked kernel reads them otherwise
cudaError_t launch_adj5(const AdjArgs& a, const Tile& t, int K, int ut, cudaStream_t s)
{
    if (!v3_fits(a.g, K) || !v5_supported(a.g.dims, K, t)) return cudaErrorInvalidValue;
    if (ut != U_FP32) {
        Tile t3 = t;
        t3.ver = 3;
        t3.pf = 0;
        return launch_adj3(a, t3, K, ut, s);
    }
    AdjArgs b = a;
    b.zlen = t.zlen;
    switch (K) {
    case 1: return adj5_k<1>(b, t, s);
    case 2: return adj5_k<2>(b, t, s);
    case 4: return adj5_k<4>(b, t, s);
    case 8: return adj5_k<8>(b, t, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ckfwi

namespace ckfwi {

cudaError_t launch_fwd5_batch(const BatchLaunch<FwdArgs>& b, const Tile& t, int K, int ck, cudaStream_t s)
{
    if (b.dims != 3 || b.lanes < 1 || b.blocks < 1 || b.blocks > 0x7fffffffLL || !v5_supported(3, K, t))
        return cudaErrorInvalidValue;
    const bool two = t.pf == 2;
    switch (K) {
    case 1: return two ? fwd5b_go<1, 2>(b, ck, s) : fwd5b_go<1, 1>(b, ck, s);
    case 2: return two ? fwd5b_go<2, 2>(b, ck, s) : fwd5b_go<2, 1>(b, ck, s);
    case 4: return two ? fwd5b_go<4, 2>(b, ck, s) : fwd5b_go<4, 1>(b, ck, s);
    case 8: return two ? fwd5b_go<8, 2>(b, ck, s) : fwd5b_go<8, 1>(b, ck, s);
    default: return cudaErrorInvalidValue;
    }
}

// FP32 u^{j-1} only (16-bit batches read through the vector-blocked kernel)
cudaError_t launch_adj5_batch(const BatchLaunch<AdjArgs>& b, const Tile& t, int K, int ut, cudaStream_t s)
{
    if (b.dims != 3 || b.lanes < 1 || b.blocks < 1 || b.blocks > 0x7fffffffLL || !v5_supported(3, K, t))
        return cudaErrorInvalidValue;
    if (ut != U_FP32) {
        Tile t3 = t;
        t3.ver = 3;
        t3.pf = 0;
        return launch_adj3_batch(b, t3, K, ut, s);
    }
    const bool two = t.pf == 2;
    switch (K) {
    case 1: return two ? adj5b_go<1, 2>(b, s) : adj5b_go<1, 1>(b, s);
    case 2: return two ? adj5b_go<2, 2>(b, s) : adj5b_go<2, 1>(b, s);
    case 4: return two ? adj5b_go<4, 2>(b, s) : adj5b_go<4, 1>(b, s);
    case 8: return two ? adj5b_go<8, 2>(b, s) : adj5b_go<8, 1>(b, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ckfwi
