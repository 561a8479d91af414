// Forward OT2 step with a compile-time z queue and ring (3D, orders 2-8,
// Tile.ver 8).
//
// The async-copy forward step (stencil_v4.cu) spends about a quarter of its
// instructions moving the register queue of z neighbours down by one plane
// and computing ring slots and copy addresses every plane.  Here the plane
// loop is unrolled by the queue length 2K+1, and the ring of u tiles has the
// same length (prefetch depth D = K: tiles z .. z+2K in flight), so for the
// n-th plane of an unrolled round every queue index and every ring slot is a
// compile-time constant: no queue moves, no slot arithmetic, every shared
// load [register + immediate].  The point fields (u^{n-1}, w) come straight
// from global memory into registers one plane ahead.  The arithmetic is
// lap3's difference-form Laplacian and leap2v's increment-form update in
// their order, so the values are bitwise those of every other generation.
//
// Plane z = z0 + 9 r + ph (K = 4; 2K+1 = 9 in general):
//   queue:  plane z + d (|d| <= K) in q[(ph + d) mod (2K+1)]
//   ring:   the tile of plane p in slot (p - z0) mod (2K+1)
//   groups: one commit group per tile; tile p is group p - z0
// Step z: wait until at most D - 1 groups are pending (tile z+K has landed),
// barrier, issue tile z+K+D into the slot of plane z-1, take the queue's
// new plane z+K from its tile, compute plane z.
#include <utility>

#include "stencil_v3.cuh"

namespace ckfwi {
namespace {

constexpr int V6 = 4;
constexpr int TX6 = 8;
constexpr int TY6 = 16;

template <int K>
struct G6 {
    using G = G3<K, V6, TX6, TY6>;
    static constexpr int NQ = 2 * K + 1;                // queue length = ring length
    static constexpr int D = K;                         // planes of prefetch
    static constexpr int NT = TX6 * TY6;
    static constexpr int NXH = 2 * TY6 * (G::PX / V6);
    static constexpr int NYH = 2 * K * (G::BXP / V6);
    static constexpr int NH = NXH + NYH;
    static constexpr int HPT = (NH + NT - 1) / NT;
    static constexpr unsigned TB = G::TILE * 4u;        // bytes of a u tile
};

__device__ __forceinline__ unsigned su32_6(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16_6(unsigned dst, const float* src, unsigned n)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void commit6() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void wait6() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// a thread's copies of a u tile, described once (see Desc5 in stencil_v5.cu)
template <int K>
struct Desc6 {
    using H = G6<K>;
    using G = typename H::G;
    unsigned cd, cn;
    int cs;
    unsigned hd[H::HPT], hn[H::HPT];
    int hs[H::HPT];
    bool hon[H::HPT];
    __device__ __forceinline__ void init(int tid, int tx, int ty, int xb, int yb, int nx, int ny, int px)
    {
        const int x0 = xb + V6 * tx, y = yb + ty;
        const bool cv = y < ny && x0 < nx;
        cd = 4u * (unsigned)((ty + K) * G::RX + G::PX + V6 * tx);
        cs = cv ? y * px + x0 : 0;
        cn = cv ? 16u : 0u;
#pragma unroll
        for (int k = 0; k < H::HPT; ++k) {
            const int h = tid + k * H::NT;
            bool v = false;
            int off = 0, so = 0;
            hon[k] = h < H::NH;
            if (h < H::NXH) {
                constexpr int PV = G::PX / V6;
                const int side = h / (TY6 * PV), rem = h % (TY6 * PV);
                const int r = rem / PV, c = rem % PV;
                const int yy = yb + r;
                const int xx = (side ? xb + G::BXP : xb - G::PX) + c * V6;
                v = yy < ny && (side == 0 || xb + G::BXP < nx + K);
                off = yy * px + xx;
                so = (r + K) * G::RX + (side ? G::PX + G::BXP : 0) + c * V6;
            } else if (h < H::NH) {
                constexpr int BV = G::BXP / V6;
                const int h2 = h - H::NXH;
                const int side = h2 / (K * BV), rem = h2 % (K * BV);
                const int rr = rem / BV, c = rem % BV;
                const int yy = side ? yb + TY6 + rr : yb - K + rr;
                const int xx = xb + c * V6;
                v = xx < nx && (side == 0 || yy < ny + K);
                off = yy * px + xx;
                so = (side ? TY6 + K + rr : rr) * G::RX + G::PX + c * V6;
            }
            hd[k] = 4u * (unsigned)so;
            hs[k] = v ? off : 0;
            hn[k] = v ? 16u : 0u;
        }
    }
    __device__ __forceinline__ void tile(unsigned slot, const float* pl) const
    {
        cp16_6(slot + cd, pl + cs, cn);
#pragma unroll
        for (int k = 0; k < H::HPT; ++k)
            if (hon[k]) cp16_6(slot + hd[k], pl + hs[k], hn[k]);
    }
};

// lap3's Laplacian at phase PH: the plane z + d of the window sits in
// q[(PH + d) mod NQ]; the staged tile of plane z at `sm`.
template <int K, int PH>
__device__ __forceinline__ void lap6(float (&out)[V6], const float (&q)[2 * K + 1][V6], const float* sm, int tx,
                                     int ty, const float2 (&cj2)[K + 1])
{
    using G = G3<K, V6, TX6, TY6>;
    constexpr int NQ = 2 * K + 1;
    const int r = ty + K;
    float xw[V6 + 2 * G::PX];
#pragma unroll
    for (int k = 0; k < G::NW; ++k) {
        float t[V6];
        sld<V6>(t, sm + r * G::RX + V6 * tx + V6 * k);
#pragma unroll
        for (int i = 0; i < V6; ++i) xw[V6 * k + i] = t[i];
    }
    const float* u = q[PH % NQ];
    float2 nu[V6 / 2], acc[V6 / 2];
#pragma unroll
    for (int p = 0; p < V6 / 2; ++p) {
        nu[p] = f2(-u[2 * p], -u[2 * p + 1]);
        acc[p] = f2(0.0f, 0.0f);
    }
#pragma unroll
    for (int j = K; j >= 1; --j) {
        float yp[V6], ym[V6];
        sld<V6>(yp, sm + (r + j) * G::RX + G::PX + V6 * tx);
        sld<V6>(ym, sm + (r - j) * G::RX + G::PX + V6 * tx);
        const float* zp = q[(PH + j) % NQ];
        const float* zm = q[(PH - j + NQ) % NQ];
#pragma unroll
        for (int p = 0; p < V6 / 2; ++p) {
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
    for (int p = 0; p < V6 / 2; ++p) {
        out[2 * p] = acc[p].x;
        out[2 * p + 1] = acc[p].y;
    }
}

template <int K, int CK>
struct Fwd6 {
    using H = G6<K>;
    using G = typename H::G;
    static constexpr int NQ = H::NQ;
    static constexpr int D = H::D;

    // one plane of an unrolled round, at compile-time phase PH
    template <int PH>
    __device__ __forceinline__ static void step(const FwdArgs& a, float (&q)[NQ][V6], float (&upc)[V6],
                                                float (&wc)[V6], float (&upn)[V6], float (&wn)[V6],
                                                const float* ring, unsigned ub, const Desc6<K>& d, int z, int z1,
                                                int zumax, long long pxy, long long col, bool cload, bool full,
                                                int x0, int nx, int tx, int ty, const float2 (&cj2)[K + 1],
                                                const float (&ecol)[V6], const Inj3<V6>& ij)
    {
        wait6<D - 1>();
        __syncthreads();
        // tile z+K+D into the slot of plane z-1
        d.tile(ub + ((PH + K + D) % NQ) * H::TB, a.u + (long long)min(z + K + D, zumax) * pxy);
        commit6();
        // the point fields of plane z+1 into registers
        if (cload) {
            const long long po = (long long)min(z + 1, z1 - 1) * pxy + col;
            gld<V6>(upn, a.up + po);
            gld<V6>(wn, a.w + po);
        }
        // the queue's new plane z+K from its tile
        sld<V6>(q[(PH + K) % NQ], ring + ((PH + K) % NQ) * G::TILE + d.cd / 4);
        if (cload) {
            const float* uc = q[PH % NQ];
            float s[V6];
            lap6<K, PH>(s, q, ring + (PH % NQ) * G::TILE, tx, ty, cj2);
            ij.add(s, a.src, z);
            const float ez = a.eta[z];
            float v[V6];
#pragma unroll
            for (int p = 0; p < V6 / 2; ++p) {
                const int i = 2 * p;
                const float2 eta = __fadd2_rn(f2(ez, ez), f2(ecol[i], ecol[i + 1]));
                const float2 r = leap2v(f2(uc[i], uc[i + 1]), f2(upc[i], upc[i + 1]), f2(wc[i], wc[i + 1]),
                                        f2(s[i], s[i + 1]), eta, a.hdt);
                v[i] = r.x;
                v[i + 1] = r.y;
            }
            const long long o = (long long)z * pxy + col;
            if (full) {
                vst<V6>(a.out + o, v);
                if (CK == CK_FP32) vstp<V6>(static_cast<float*>(a.ck_up) + o, uc);
            } else {
#pragma unroll
                for (int i = 0; i < V6; ++i) {
                    if (x0 + i < nx) {
                        a.out[o + i] = v[i];
                        if (CK == CK_FP32) static_cast<float*>(a.ck_up)[o + i] = uc[i];
                    }
                }
            }
            if (CK == CK_BF16) {
                st16<__nv_bfloat16, V6>(a.ck_u, o, v, full, x0, nx);
                st16<__nv_bfloat16, V6>(a.ck_up, o, uc, full, x0, nx);
            } else if (CK == CK_FP16) {
                const bool inf = st16<__half, V6>(a.ck_u, o, v, full, x0, nx) | st16<__half, V6>(a.ck_up, o, uc, full, x0, nx);
                if (inf) atomicOr(a.err, 1);
            }
        }
#pragma unroll
        for (int i = 0; i < V6; ++i) {
            upc[i] = upn[i];
            wc[i] = wn[i];
        }
    }

    template <int... PH>
    __device__ __forceinline__ static void round(std::integer_sequence<int, PH...>, const FwdArgs& a,
                                                 float (&q)[NQ][V6], float (&upc)[V6], float (&wc)[V6],
                                                 float (&upn)[V6], float (&wn)[V6], const float* ring, unsigned ub,
                                                 const Desc6<K>& d, int zr, int z1, int zumax, long long pxy,
                                                 long long col, bool cload, bool full, int x0, int nx, int tx, int ty,
                                                 const float2 (&cj2)[K + 1], const float (&ecol)[V6],
                                                 const Inj3<V6>& ij)
    {
        // planes zr + PH in order, stopping at z1 (the same for every thread of the CTA)
        bool go = true;
        ((go = go && zr + PH < z1,
          go ? step<PH>(a, q, upc, wc, upn, wn, ring, ub, d, zr + PH, z1, zumax, pxy, col, cload, full, x0, nx, tx, ty,
                        cj2, ecol, ij)
             : void()),
         ...);
    }
};

template <int K, int CK>
__device__ __forceinline__ void fwd6_body(const FwdArgs& a, float* smem, int bxi, int byi, int bzi, int gxn, int gyn)
{
    using F = Fwd6<K, CK>;
    using H = G6<K>;
    using G = typename H::G;
    constexpr int NQ = H::NQ;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX6 + tx;
    const int nz = a.g.nz, ny = a.g.ny, nx = a.g.nx;
    const int px = (int)a.g.px;
    const long long pxy = a.g.pxy;
    const int xb = bxi * G::BXP, yb = byi * TY6;
    const int x0 = xb + V6 * tx;
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
    const bool full = rowact && x0 + V6 <= nx;
    const long long col = (long long)y * px + x0;
    float ecol[V6];
#pragma unroll
    for (int i = 0; i < V6; ++i)
        ecol[i] = (rowact && x0 + i < nx) ? __fadd_rn(a.eta[nz + y], a.eta[nz + ny + x0 + i]) : 0.0f;
    float2 cj2[K + 1];
#pragma unroll
    for (int j = 0; j <= K; ++j) cj2[j] = f2(a.c[j], a.c[j]);
    Inj3<V6> ij;
    ij.init(a.src, y, x0, nx, rowact);
    Desc6<K> d;
    d.init(tid, tx, ty, xb, yb, nx, ny, px);
    const unsigned ub = su32_6(smem);
    const int zumax = nz + K - 1;

    // queue: planes z0 - K .. z0 - 1 straight from global memory (q[(d + NQ) mod NQ])
    float q[NQ][V6];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        if (cload) gld<V6>(q[NQ - K + i], a.u + (long long)(z0 - K + i) * pxy + col);
        else vzero<V6>(q[NQ - K + i]);
    }
    // prologue: tiles z0 .. z0 + K + D - 1, one group each
#pragma unroll 1
    for (int p = 0; p < K + H::D; ++p) {
        d.tile(ub + p * H::TB, a.u + (long long)min(z0 + p, zumax) * pxy);
        commit6();
    }
    float upc[V6], wc[V6], upn[V6], wn[V6];
    if (cload) {
        gld<V6>(upc, a.up + (long long)z0 * pxy + col);
        gld<V6>(wc, a.w + (long long)z0 * pxy + col);
    } else {
        vzero<V6>(upc);
        vzero<V6>(wc);
    }
    vzero<V6>(upn);
    vzero<V6>(wn);
    // the queue's planes z0 .. z0 + K - 1 from tiles 0 .. K-1
    wait6<H::D>();
    __syncthreads();
#pragma unroll
    for (int i = 0; i < K; ++i) sld<V6>(q[i], smem + i * G::TILE + d.cd / 4);

    for (int zr = z0; zr < z1; zr += NQ)
        F::round(std::make_integer_sequence<int, NQ>{}, a, q, upc, wc, upn, wn, smem, ub, d, zr, z1, zumax, pxy, col,
                 cload, full, x0, nx, tx, ty, cj2, ecol, ij);
    wait6<0>();      // no copy may land after the CTA has left
}

// 2K+1 tiles of 3.84 KB at order 8 (35 KB a CTA): four CTAs an SM at <= 128 registers
template <int K, int CK>
__global__ void __launch_bounds__(TX6 * TY6, 4) fwd6_kernel(const FwdArgs a)
{
    extern __shared__ __align__(16) float smem6[];
    fwd6_body<K, CK>(a, smem6, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y);
}

template <int K>
cudaError_t fwd6_go(const FwdArgs& a, int ck, cudaStream_t s)
{
    using G = typename G6<K>::G;
    const dim3 blk(TX6, TY6, 1);
    const dim3 grd((a.g.nx + G::BXP - 1) / G::BXP, (a.g.ny + TY6 - 1) / TY6, (a.g.nz + a.zlen - 1) / a.zlen);
    const size_t sh = (size_t)G6<K>::NQ * G6<K>::TB;
    cudaError_t e = cudaSuccess;
    switch (ck) {
    case CK_NONE:
        e = cudaFuncSetAttribute(fwd6_kernel<K, CK_NONE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        if (e == cudaSuccess) fwd6_kernel<K, CK_NONE><<<grd, blk, sh, s>>>(a);
        break;
    case CK_FP32:
        e = cudaFuncSetAttribute(fwd6_kernel<K, CK_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        if (e == cudaSuccess) fwd6_kernel<K, CK_FP32><<<grd, blk, sh, s>>>(a);
        break;
    case CK_BF16:
        e = cudaFuncSetAttribute(fwd6_kernel<K, CK_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        if (e == cudaSuccess) fwd6_kernel<K, CK_BF16><<<grd, blk, sh, s>>>(a);
        break;
    case CK_FP16:
        e = cudaFuncSetAttribute(fwd6_kernel<K, CK_FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        if (e == cudaSuccess) fwd6_kernel<K, CK_FP16><<<grd, blk, sh, s>>>(a);
        break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

bool v6_supported(int dims, int K, const Tile& t)
{
    return dims == 3 && t.ver == 8 && t.zlen >= 1 && (K == 1 || K == 2 || K == 4) && t.bx == V6 * TX6 &&
           t.by == TY6 && t.vec == V6;
}

cudaError_t launch_fwd6(const FwdArgs& a, const Tile& t, int K, int ck, cudaStream_t s)
{
    FwdArgs b = a;
    b.zlen = t.zlen;
    if (!v3_fits(a.g, K) || !v6_supported(a.g.dims, K, t)) return cudaErrorInvalidValue;
    switch (K) {
    case 1: return fwd6_go<1>(b, ck, s);
    case 2: return fwd6_go<2>(b, ck, s);
    case 4: return fwd6_go<4>(b, ck, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ckfwi
