// Forward and fused reverse steps with every global load as an asynchronous
// copy into shared-memory rings (3D, fourth kernel generation).
//
// The vector-blocked kernel (stencil_v3.cuh) holds the next plane's values,
// halos and point fields in registers, one plane ahead; at 128 registers a
// thread, an SM keeps 16 warps and the kernel waits on global loads.  Here
// the same arithmetic (lap3, leap2v) reads
//   * the halo'd u tile of plane z from a ring of K + D + 1 tiles,
//   * u^{n-1} and w of plane z from rings of D + 1 point tiles,
//   * the z queue's new plane z + K from the u ring (one shared load),
// and every thread issues cp.async copies D planes ahead: its own vector of
// the u tile, at most two halo vectors, and its vectors of u^{n-1} and w.
// Copies that fall outside the needed region are zero-filled (source size
// 0), so the halo and ragged-edge rules are those of the other kernels and
// the results bitwise theirs.  No prefetch registers: about a hundred
// registers a thread and deeper prefetch.
//
// Step t (plane z = z0 + t): wait until at most D - 1 copy groups are in
// flight (the group of u plane z + K is complete), barrier, issue the group
// of u plane z + K + D and point planes z + D into the slots freed by step
// t - 1, compute plane z.
#include "stencil_v3.cuh"

namespace ckfwi {
namespace {

template <int K, int V, int TX, int TY, int PF>
struct G4 {
    using G = G3<K, V, TX, TY>;
    static constexpr int D = PF;                   // planes of prefetch
    static constexpr int RU = K + D + 1;           // u tiles in the ring
    static constexpr int RP = D + 1;               // point planes in each point ring
    static constexpr int PT = G::BXP * TY;         // floats of a point tile
    static constexpr int NT = TX * TY;             // threads
    static constexpr int NXH = 2 * TY * (G::PX / V);      // x-halo vectors of a u tile
    static constexpr int NYH = 2 * K * (G::BXP / V);      // y-halo vectors
    static constexpr int NH = NXH + NYH;
    static constexpr int HPT = (NH + NT - 1) / NT;        // halo vectors per thread
    static constexpr size_t FLOATS = (size_t)RU * G::TILE + 2 * (size_t)RP * PT;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// V floats from global to shared, asynchronously; zero-filled when !valid
template <int V>
__device__ __forceinline__ void cp_async(float* dst, const float* src, bool valid)
{
    const unsigned n = valid ? 4u * V : 0u;
    if constexpr (V == 4)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(n)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(n)
                     : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// One thread's share of a plane's copies: its u-tile vector, its halo
// vectors, its point vectors.  Offsets are element offsets from the plane's
// origin (add z * pxy); a copy whose source is not needed is zero-filled and
// points at the plane origin instead (never read).
template <int K, int V, int TX, int TY, int PF>
struct Copies4 {
    using G = G3<K, V, TX, TY>;
    using H = G4<K, V, TX, TY, PF>;
    int cg, cs;                    // centre: global offset, shared offset in a u tile
    bool cv;
    int hg[H::HPT], hs[H::HPT];    // halo vectors
    bool hv[H::HPT], hon[H::HPT];  // needed; the thread has this halo vector at all
    int ps;                        // point tile shared offset
    __device__ __forceinline__ void init(int tid, int tx, int ty, int xb, int yb, int nx, int ny, int px)
    {
        const int x0 = xb + V * tx, y = yb + ty;
        cv = y < ny && x0 < nx;
        cg = y * px + x0;
        cs = (ty + K) * G::RX + G::PX + V * tx;
        ps = ty * G::BXP + V * tx;
#pragma unroll
        for (int k = 0; k < H::HPT; ++k) {
            const int h = tid + k * H::NT;
            hv[k] = false;
            hon[k] = h < H::NH;
            hg[k] = 0;
            hs[k] = 0;
            if (h < H::NXH) {
                constexpr int PV = G::PX / V;                   // vectors per halo row
                const int side = h / (TY * PV), rem = h % (TY * PV);
                const int r = rem / PV, c = rem % PV;
                const int yy = yb + r;
                const int xx = (side ? xb + G::BXP : xb - G::PX) + c * V;
                hv[k] = yy < ny && (side == 0 || xb + G::BXP < nx + K);
                hg[k] = yy * px + xx;
                hs[k] = (r + K) * G::RX + (side ? G::PX + G::BXP : 0) + c * V;
            } else if (h < H::NH) {
                constexpr int BV = G::BXP / V;                  // vectors per halo row
                const int h2 = h - H::NXH;
                const int side = h2 / (K * BV), rem = h2 % (K * BV);
                const int rr = rem / BV, c = rem % BV;
                const int yy = side ? yb + TY + rr : yb - K + rr;
                const int xx = xb + c * V;
                hv[k] = xx < nx && (side == 0 || yy < ny + K);
                hg[k] = yy * px + xx;
                hs[k] = (side ? TY + K + rr : rr) * G::RX + G::PX + c * V;
            }
        }
    }
    // the u tile of the plane at offset zoff (valid: the plane is needed)
    __device__ __forceinline__ void tile(float* slot, const float* u, int zoff, bool plane) const
    {
        cp_async<V>(slot + cs, cv && plane ? u + zoff + cg : u, cv && plane);
#pragma unroll
        for (int k = 0; k < H::HPT; ++k)
            if (hon[k]) cp_async<V>(slot + hs[k], hv[k] && plane ? u + zoff + hg[k] : u, hv[k] && plane);
    }
    __device__ __forceinline__ void point(float* slot, const float* f, int zoff, bool plane) const
    {
        cp_async<V>(slot + ps, cv && plane ? f + zoff + cg : f, cv && plane);
    }
};

template <int K, int V, int TX, int TY, int PF, int CK>
__device__ __forceinline__ void fwd4_body(const FwdArgs& a, float* smem, int bxi, int byi, int bzi, int gxn,
                                          int gyn)
{
    using G = G3<K, V, TX, TY>;
    using H = G4<K, V, TX, TY, PF>;
    constexpr int D = H::D;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int nz = a.g.nz, ny = a.g.ny, nx = a.g.nx;
    const int px = (int)a.g.px, pxy = (int)a.g.pxy;
    const int xb = bxi * G::BXP, yb = byi * TY;
    const int x0 = xb + V * tx;
    const int y = yb + ty;

    if (a.smp.n > 0) {   // receiver sampling of u^n by the first threads of the grid
        const int gt = ((bzi * gyn + byi) * gxn + bxi) * (TX * TY) + tid;
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
    const bool full = rowact && x0 + V <= nx;
    const int col = y * px + x0;
    float ecol[V];
#pragma unroll
    for (int i = 0; i < V; ++i)
        ecol[i] = (rowact && x0 + i < nx) ? __fadd_rn(a.eta[nz + y], a.eta[nz + ny + x0 + i]) : 0.0f;
    Inj3<V> ij;
    ij.init(a.src, y, x0, nx, rowact);
    Copies4<K, V, TX, TY, PF> cp;
    cp.init(tid, tx, ty, xb, yb, nx, ny, px);

    float* ring = smem;                          // RU u tiles
    float* upr = smem + H::RU * G::TILE;         // RP point tiles of u^{n-1}
    float* wr = upr + H::RP * H::PT;             // RP point tiles of w
    const int zqmax = nz + K - 1;

    // queue planes z0 - K .. z0 - 1 straight into registers
    float q[2 * K + 1][V];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        if (cload) gld<V>(q[i], a.u + (z0 - K + i) * pxy + col);
        else vzero<V>(q[i]);
    }
    // prologue: u planes z0 .. z0 + K + D - 1 and point planes z0 .. z0 + D - 1,
    // one copy group per plane index; plane p's u tile sits in slot (p - z0) % RU
#pragma unroll 1
    for (int p = 0; p < K + D; ++p) {
        const int zu = z0 + p;
        cp.tile(ring + p * G::TILE, a.u, min(zu, zqmax) * pxy, zu <= zqmax);
        if (p < D) {
            const int zp = z0 + p;
            cp.point(upr + p * H::PT, a.up, min(zp, z1 - 1) * pxy, zp < z1);
            cp.point(wr + p * H::PT, a.w, min(zp, z1 - 1) * pxy, zp < z1);
        }
        cp_commit();
    }
    // the queue's planes z0 .. z0 + K - 1 come from the ring once they land
    cp_wait<D>();
    __syncthreads();
#pragma unroll
    for (int i = 0; i < K; ++i) sld<V>(q[K + i], ring + i * G::TILE + cp.cs);

    int su = 0, sp = 0;                          // ring slots of plane z
    for (int z = z0; z < z1; ++z) {
        // group of u plane z + K complete in every thread
        cp_wait<D - 1>();
        __syncthreads();
        // refill the slots step z - 1 freed: u plane z + K + D, point plane z + D
        {
            const int zu = z + K + D, zp = z + D;
            int sn = su + K + D;
            if (sn >= H::RU) sn -= H::RU;
            int pn = sp + D;
            if (pn >= H::RP) pn -= H::RP;
            cp.tile(ring + sn * G::TILE, a.u, min(zu, zqmax) * pxy, zu <= zqmax);
            cp.point(upr + pn * H::PT, a.up, min(zp, z1 - 1) * pxy, zp < z1);
            cp.point(wr + pn * H::PT, a.w, min(zp, z1 - 1) * pxy, zp < z1);
            cp_commit();
        }
        int sk = su + K;
        if (sk >= H::RU) sk -= H::RU;
        sld<V>(q[2 * K], ring + sk * G::TILE + cp.cs);
        const float* sm = ring + su * G::TILE;
        if (cload) {
            float upv[V], wv[V];
            sld<V>(upv, upr + sp * H::PT + cp.ps);
            sld<V>(wv, wr + sp * H::PT + cp.ps);
            const float* uc = q[K];
            float s[V];
            lap3<K, V, TX, TY>(s, q, sm, tx, ty, a.c);
            ij.add(s, a.src, z);
            const float ez = a.eta[z];
            float v[V];
#pragma unroll
            for (int p = 0; p < V / 2; ++p) {
                const int i = 2 * p;
                const float2 eta = __fadd2_rn(f2(ez, ez), f2(ecol[i], ecol[i + 1]));
                const float2 r = leap2v(f2(uc[i], uc[i + 1]), f2(upv[i], upv[i + 1]), f2(wv[i], wv[i + 1]),
                                        f2(s[i], s[i + 1]), eta, a.hdt);
                v[i] = r.x;
                v[i + 1] = r.y;
            }
            const long long o = (long long)z * pxy + col;
            if (full) {
                vst<V>(a.out + o, v);
                if (CK == CK_FP32) vstp<V>(static_cast<float*>(a.ck_up) + o, uc);
            } else {
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    if (x0 + i < nx) {
                        a.out[o + i] = v[i];
                        if (CK == CK_FP32) static_cast<float*>(a.ck_up)[o + i] = uc[i];
                    }
                }
            }
            if (CK == CK_BF16) {
                st16<__nv_bfloat16, V>(a.ck_u, o, v, full, x0, nx);
                st16<__nv_bfloat16, V>(a.ck_up, o, uc, full, x0, nx);
            } else if (CK == CK_FP16) {
                const bool inf = st16<__half, V>(a.ck_u, o, v, full, x0, nx) | st16<__half, V>(a.ck_up, o, uc, full, x0, nx);
                if (inf) atomicOr(a.err, 1);
            }
        }
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) {
#pragma unroll
            for (int k = 0; k < V; ++k) q[i][k] = q[i + 1][k];
        }
        if (++su == H::RU) su = 0;
        if (++sp == H::RP) sp = 0;
    }
    cp_wait<0>();     // no copy may land after the CTA has left
}

// One plane of prefetch needs 31 KB of shared memory per 128-thread CTA at
// order 8 (two planes: 39 KB, five CTAs per SM); capped at 80 registers
// (no spill up to order 8), six CTAs fit.
template <int K, int V, int PF>
constexpr int fwd4_min_blocks() { return V == 4 && PF == 1 && K <= 4 ? 6 : 1; }

template <int K, int V, int TX, int TY, int PF, int CK>
__global__ void __launch_bounds__(TX * TY, fwd4_min_blocks<K, V, PF>()) fwd4_kernel(const FwdArgs a)
{
    extern __shared__ __align__(16) float smem4[];
    fwd4_body<K, V, TX, TY, PF, CK>(a, smem4, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y);
}

template <int K, int V, int TX, int TY, int PF>
cudaError_t fwd4_go(const FwdArgs& a, int ck, cudaStream_t s)
{
    using G = G3<K, V, TX, TY>;
    using H = G4<K, V, TX, TY, PF>;
    const dim3 blk(TX, TY, 1);
    const dim3 grd((a.g.nx + G::BXP - 1) / G::BXP, (a.g.ny + TY - 1) / TY, (a.g.nz + a.zlen - 1) / a.zlen);
    const size_t sh = H::FLOATS * sizeof(float);
    cudaError_t e = cudaSuccess;
    switch (ck) {
    case CK_NONE:
        e = cudaFuncSetAttribute(fwd4_kernel<K, V, TX, TY, PF, CK_NONE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        if (e == cudaSuccess) fwd4_kernel<K, V, TX, TY, PF, CK_NONE><<<grd, blk, sh, s>>>(a);
        break;
    case CK_FP32:
        e = cudaFuncSetAttribute(fwd4_kernel<K, V, TX, TY, PF, CK_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        if (e == cudaSuccess) fwd4_kernel<K, V, TX, TY, PF, CK_FP32><<<grd, blk, sh, s>>>(a);
        break;
    case CK_BF16:
        e = cudaFuncSetAttribute(fwd4_kernel<K, V, TX, TY, PF, CK_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        if (e == cudaSuccess) fwd4_kernel<K, V, TX, TY, PF, CK_BF16><<<grd, blk, sh, s>>>(a);
        break;
    case CK_FP16:
        e = cudaFuncSetAttribute(fwd4_kernel<K, V, TX, TY, PF, CK_FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        if (e == cudaSuccess) fwd4_kernel<K, V, TX, TY, PF, CK_FP16><<<grd, blk, sh, s>>>(a);
        break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int K>
cudaError_t fwd4_k(const FwdArgs& a, const Tile& t, int ck, cudaStream_t s)
{
    if (t.vec == 4 && t.bx == 32 && t.by == 16 && t.pf == 1) return fwd4_go<K, 4, 8, 16, 1>(a, ck, s);
    if (t.vec == 4 && t.bx == 32 && t.by == 16) return fwd4_go<K, 4, 8, 16, 2>(a, ck, s);
    if (t.vec == 2 && t.bx == 32 && t.by == 16) return fwd4_go<K, 2, 16, 16, 2>(a, ck, s);
    return cudaErrorInvalidValue;
}


// Fused reverse step, same structure: rings of lam^j and u^{j-1} tiles and
// of lam^{j+1}, w and gacc point tiles; u^{j-1} in FP32 only (16-bit
// checkpoint reads use the vector-blocked kernel).
template <int K, int V, int TX, int TY, int PF>
__device__ __forceinline__ void adj4_body(const AdjArgs& a, float* smem, int bxi, int byi, int bzi)
{
    using G = G3<K, V, TX, TY>;
    using H = G4<K, V, TX, TY, PF>;
    constexpr int D = H::D;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int nz = a.g.nz, ny = a.g.ny, nx = a.g.nx;
    const int px = (int)a.g.px, pxy = (int)a.g.pxy;
    const int xb = bxi * G::BXP, yb = byi * TY;
    const int x0 = xb + V * tx;
    const int y = yb + ty;
    const int z0 = bzi * a.zlen;
    if (z0 >= nz) return;
    const int z1 = min(z0 + a.zlen, nz);
    const bool rowact = y < ny;
    const bool cload = rowact && x0 < nx;
    const bool full = rowact && x0 + V <= nx;
    const int col = y * px + x0;
    float ecol[V];
#pragma unroll
    for (int i = 0; i < V; ++i)
        ecol[i] = (rowact && x0 + i < nx) ? __fadd_rn(a.eta[nz + y], a.eta[nz + ny + x0 + i]) : 0.0f;
    Inj3<V> ia, is;
    ia.init(a.adj, y, x0, nx, rowact);
    is.init(a.src, y, x0, nx, rowact);
    Copies4<K, V, TX, TY, PF> cp;
    cp.init(tid, tx, ty, xb, yb, nx, ny, px);
    const float* uu = static_cast<const float*>(a.u);

    float* lring = smem;                              // RU lam^j tiles
    float* uring = lring + H::RU * G::TILE;           // RU u^{j-1} tiles
    float* l2r = uring + H::RU * G::TILE;             // RP point tiles each
    float* wr = l2r + H::RP * H::PT;
    float* gr = wr + H::RP * H::PT;
    const int zqmax = nz + K - 1;

    float ql[2 * K + 1][V], qu[2 * K + 1][V];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const int o = (z0 - K + i) * pxy + col;
        if (cload) {
            gld<V>(ql[i], a.l1 + o);
            gld<V>(qu[i], uu + o);
        } else {
            vzero<V>(ql[i]);
            vzero<V>(qu[i]);
        }
    }
#pragma unroll 1
    for (int p = 0; p < K + D; ++p) {
        const int zu = z0 + p;
        cp.tile(lring + p * G::TILE, a.l1, min(zu, zqmax) * pxy, zu <= zqmax);
        cp.tile(uring + p * G::TILE, uu, min(zu, zqmax) * pxy, zu <= zqmax);
        if (p < D) {
            const int zp = z0 + p, zo = min(zp, z1 - 1) * pxy;
            cp.point(l2r + p * H::PT, a.l2, zo, zp < z1);
            cp.point(wr + p * H::PT, a.w, zo, zp < z1);
            cp.point(gr + p * H::PT, a.gacc, zo, zp < z1);
        }
        cp_commit();
    }
    cp_wait<D>();
    __syncthreads();
#pragma unroll
    for (int i = 0; i < K; ++i) {
        sld<V>(ql[K + i], lring + i * G::TILE + cp.cs);
        sld<V>(qu[K + i], uring + i * G::TILE + cp.cs);
    }

    int su = 0, sp = 0;
    for (int z = z0; z < z1; ++z) {
        cp_wait<D - 1>();
        __syncthreads();
        {
            const int zu = z + K + D, zp = z + D;
            int sn = su + K + D;
            if (sn >= H::RU) sn -= H::RU;
            int pn = sp + D;
            if (pn >= H::RP) pn -= H::RP;
            const int zo = min(zu, zqmax) * pxy, po = min(zp, z1 - 1) * pxy;
            cp.tile(lring + sn * G::TILE, a.l1, zo, zu <= zqmax);
            cp.tile(uring + sn * G::TILE, uu, zo, zu <= zqmax);
            cp.point(l2r + pn * H::PT, a.l2, po, zp < z1);
            cp.point(wr + pn * H::PT, a.w, po, zp < z1);
            cp.point(gr + pn * H::PT, a.gacc, po, zp < z1);
            cp_commit();
        }
        int sk = su + K;
        if (sk >= H::RU) sk -= H::RU;
        sld<V>(ql[2 * K], lring + sk * G::TILE + cp.cs);
        sld<V>(qu[2 * K], uring + sk * G::TILE + cp.cs);
        if (cload) {
            float l2v[V], wv[V], gv[V];
            sld<V>(l2v, l2r + sp * H::PT + cp.ps);
            sld<V>(wv, wr + sp * H::PT + cp.ps);
            sld<V>(gv, gr + sp * H::PT + cp.ps);
            float sl_[V], su_[V];
            lap3<K, V, TX, TY>(sl_, ql, lring + su * G::TILE, tx, ty, a.c);
            ia.add(sl_, a.adj, z);
            lap3<K, V, TX, TY>(su_, qu, uring + su * G::TILE, tx, ty, a.c);
            is.add(su_, a.src, z);
            const float* lc = ql[K];
            const float ez = a.eta[z];
            float lam[V], gn[V];
#pragma unroll
            for (int p = 0; p < V / 2; ++p) {
                const int i = 2 * p;
                const float2 eta = __fadd2_rn(f2(ez, ez), f2(ecol[i], ecol[i + 1]));
                const float2 r = leap2v(f2(lc[i], lc[i + 1]), f2(l2v[i], l2v[i + 1]), f2(wv[i], wv[i + 1]),
                                        f2(sl_[i], sl_[i + 1]), eta, a.hdt);
                const float2 gg = __ffma2_rn(r, f2(su_[i], su_[i + 1]), f2(gv[i], gv[i + 1]));
                lam[i] = r.x;
                lam[i + 1] = r.y;
                gn[i] = gg.x;
                gn[i + 1] = gg.y;
            }
            const long long o = (long long)z * pxy + col;
            if (full) {
                vst<V>(a.l0 + o, lam);
                vst<V>(a.gacc + o, gn);
            } else {
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    if (x0 + i < nx) {
                        a.l0[o + i] = lam[i];
                        a.gacc[o + i] = gn[i];
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) {
#pragma unroll
            for (int k = 0; k < V; ++k) {
                ql[i][k] = ql[i + 1][k];
                qu[i][k] = qu[i + 1][k];
            }
        }
        if (++su == H::RU) su = 0;
        if (++sp == H::RP) sp = 0;
    }
    cp_wait<0>();
}

template <int K, int V, int TX, int TY, int PF>
__global__ void __launch_bounds__(TX * TY) adj4_kernel(const AdjArgs a)
{
    extern __shared__ __align__(16) float smem4[];
    adj4_body<K, V, TX, TY, PF>(a, smem4, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <int K, int V, int TX, int TY, int PF>
cudaError_t adj4_go(const AdjArgs& a, cudaStream_t s)
{
    using G = G3<K, V, TX, TY>;
    using H = G4<K, V, TX, TY, PF>;
    const dim3 blk(TX, TY, 1);
    const dim3 grd((a.g.nx + G::BXP - 1) / G::BXP, (a.g.ny + TY - 1) / TY, (a.g.nz + a.zlen - 1) / a.zlen);
    const size_t sh = ((size_t)2 * H::RU * G::TILE + (size_t)3 * H::RP * H::PT) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(adj4_kernel<K, V, TX, TY, PF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sh);
    if (e != cudaSuccess) return e;
    adj4_kernel<K, V, TX, TY, PF><<<grd, blk, sh, s>>>(a);
    return cudaGetLastError();
}

template <int K>
cudaError_t adj4_k(const AdjArgs& a, const Tile& t, cudaStream_t s)
{
    if (t.vec == 4 && t.bx == 32 && t.by == 16) return adj4_go<K, 4, 8, 16, 2>(a, s);
    if (t.vec == 2 && t.bx == 32 && t.by == 16) return adj4_go<K, 2, 16, 16, 2>(a, s);
    return cudaErrorInvalidValue;
}

// Batched forward step: one launch advances every lane of a batch, lane l's
// CTAs laid out like its own single-lane grid, its arguments staged from a
// device table; the single-lane body, so the values are bitwise a
// single-shot run's.
template <int K, int V, int TX, int TY, int PF, int CK>
__global__ void __launch_bounds__(TX * TY, fwd4_min_blocks<K, V, PF>())
    fwd4_batch_kernel(const FwdArgs* __restrict__ tab, const int* __restrict__ start, int nl)
{
    using G = G3<K, V, TX, TY>;
    extern __shared__ __align__(16) float smem4[];
    __shared__ __align__(16) FwdArgs a;
    const int b = stage_args(a, tab, start, nl);
    const int gx = (a.g.nx + G::BXP - 1) / G::BXP;
    const int gy = (a.g.ny + TY - 1) / TY;
    fwd4_body<K, V, TX, TY, PF, CK>(a, smem4, b % gx, (b / gx) % gy, b / (gx * gy), gx, gy);
}

template <int K, int V, int TX, int TY, int PF, int CK>
cudaError_t fwd4b_ck(const BatchLaunch<FwdArgs>& b, cudaStream_t s)
{
    const size_t sh = G4<K, V, TX, TY, PF>::FLOATS * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(fwd4_batch_kernel<K, V, TX, TY, PF, CK>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (e != cudaSuccess) return e;
    fwd4_batch_kernel<K, V, TX, TY, PF, CK><<<dim3((unsigned)b.blocks), dim3(TX, TY), sh, s>>>(b.tab, b.start,
                                                                                               b.lanes);
    return cudaGetLastError();
}

template <int K, int V, int TX, int TY, int PF>
cudaError_t fwd4b_go(const BatchLaunch<FwdArgs>& b, int ck, cudaStream_t s)
{
    switch (ck) {
    case CK_NONE: return fwd4b_ck<K, V, TX, TY, PF, CK_NONE>(b, s);
    case CK_FP32: return fwd4b_ck<K, V, TX, TY, PF, CK_FP32>(b, s);
    case CK_BF16: return fwd4b_ck<K, V, TX, TY, PF, CK_BF16>(b, s);
    case CK_FP16: return fwd4b_ck<K, V, TX, TY, PF, CK_FP16>(b, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int K>
cudaError_t fwd4b_k(const BatchLaunch<FwdArgs>& b, const Tile& t, int ck, cudaStream_t s)
{
    if (t.vec == 4 && t.bx == 32 && t.by == 16 && t.pf == 1) return fwd4b_go<K, 4, 8, 16, 1>(b, ck, s);
    if (t.vec == 4 && t.bx == 32 && t.by == 16) return fwd4b_go<K, 4, 8, 16, 2>(b, ck, s);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_fwd4_batch(const BatchLaunch<FwdArgs>& b, const Tile& t, int K, int ck, cudaStream_t s)
{
    if (b.dims != 3 || b.lanes < 1 || b.blocks < 1 || b.blocks > 0x7fffffffLL || !v4_supported(3, K, t) || t.vec != 4)
        return cudaErrorInvalidValue;
    switch (K) {
    case 1: return fwd4b_k<1>(b, t, ck, s);
    case 2: return fwd4b_k<2>(b, t, ck, s);
    case 4: return fwd4b_k<4>(b, t, ck, s);
    case 8: return fwd4b_k<8>(b, t, ck, s);
    default: return cudaErrorInvalidValue;
    }
}

bool v4_supported(int dims, int K, const Tile& t)
{
    if (dims != 3 || t.ver != 4 || t.zlen < 1 || t.by < K) return false;
    if (K != 1 && K != 2 && K != 4 && K != 8) return false;
    // two planes of prefetch (three measured no faster on 208^3, order 8);
    // the four-point forward step also with one plane and six CTAs per SM
    return t.bx == 32 && t.by == 16 && (t.vec == 2 || t.vec == 4) && (t.pf == 0 || t.pf == 2 || (t.pf == 1 && t.vec == 4 && K <= 4));
}

// the reverse step in FP32 through the rings; 16-bit u^{j-1} through the
// vector-blocked kernel of the same shape
cudaError_t launch_adj4(const AdjArgs& a, const Tile& t, int K, int ut, cudaStream_t s)
{
    if (!v3_fits(a.g, K) || !v4_supported(a.g.dims, K, t)) return cudaErrorInvalidValue;
    if (ut != U_FP32) {
        Tile t3 = t;
        t3.ver = 3;
        return launch_adj3(a, t3, K, ut, s);
    }
    AdjArgs b = a;
    b.zlen = t.zlen;
    switch (K) {
    case 1: return adj4_k<1>(b, t, s);
    case 2: return adj4_k<2>(b, t, s);
    case 4: return adj4_k<4>(b, t, s);
    case 8: return adj4_k<8>(b, t, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fwd4(const FwdArgs& a, const Tile& t, int K, int ck, cudaStream_t s)
{
    FwdArgs b = a;
    b.zlen = t.zlen;
    if (!v3_fits(a.g, K) || !v4_supported(a.g.dims, K, t)) return cudaErrorInvalidValue;
    switch (K) {
    case 1: return fwd4_k<1>(b, t, ck, s);
    case 2: return fwd4_k<2>(b, t, ck, s);
    case 4: return fwd4_k<4>(b, t, ck, s);
    case 8: return fwd4_k<8>(b, t, ck, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ckfwi
