// Vector-blocked forward and fused reverse steps for 3D grids: device code
// shared by the single-shot kernels (stencil_v3.cu) and the batched ones
// (batch_v3.cu).
//
// The single-point kernels (kernels.cu) spend most of their issue slots on
// per-point overhead: one scalar load, one shared store and 4K shared loads
// per point, scalar arithmetic, and a register queue that is shifted value
// by value.  Here a thread owns V = 2 or 4 consecutive x points of one row:
//   * every global access is one V-wide vector (the first interior column
//     and the row pitch are 16-byte aligned, so a vector never straddles);
//   * the x neighbours of all V points come from (V + 2 PX) / V vector
//     loads of the staged row, the y neighbours from one vector per row;
//   * the z neighbours live in a register queue of 2K + 1 vectors;
//   * the arithmetic runs on pairs of points with the packed FP32x2
//     instructions (__fadd2_rn, __ffma2_rn), each lane rounding exactly like
//     the scalar operation, so every value is bitwise the one the other
//     kernels compute (same operands, same order: lap_at and leapfrog);
//   * the staged plane is double buffered: one barrier per plane.
// The CTA covers V * TX x points by TY rows and marches down a run of zlen
// planes, prefetching the next plane while it computes the current one.
#pragma once
#include "stencil_body.cuh"

namespace ckfwi {
namespace {

template <int K, int V, int TX, int TY>
struct G3 {
    static constexpr int PX = K <= 4 ? 4 : 8;     // staged x-halo columns (>= K, whole vectors)
    static constexpr int BXP = V * TX;            // x points of a CTA
    static constexpr int RX = 2 * PX + BXP;       // staged row length
    static constexpr int RY = TY + 2 * K;         // staged rows
    static constexpr int TILE = RX * RY;
    static constexpr int NW = (V + 2 * PX) / V;   // vector loads of one thread's x window
    static_assert(TY >= K, "the y halo rows are staged by the first K rows of threads");
    static_assert(V == 2 || V == 4, "vector width");
};

// --------------------------------------------------------------- vectors
template <int V>
__device__ __forceinline__ void gld(float (&d)[V], const float* p)
{
    if constexpr (V == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(p));
        d[0] = t.x; d[1] = t.y; d[2] = t.z; d[3] = t.w;
    } else {
        const float2 t = __ldg(reinterpret_cast<const float2*>(p));
        d[0] = t.x; d[1] = t.y;
    }
}

template <int V>
__device__ __forceinline__ void gld_plain(float (&d)[V], const float* p)
{
    if constexpr (V == 4) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        d[0] = t.x; d[1] = t.y; d[2] = t.z; d[3] = t.w;
    } else {
        const float2 t = *reinterpret_cast<const float2*>(p);
        d[0] = t.x; d[1] = t.y;
    }
}

// a 16-bit pattern of element type UT as a float (exact for both types)
template <class UT> __device__ __forceinline__ float f16_bits(unsigned int b);
template <> __device__ __forceinline__ float f16_bits<__half>(unsigned int b) { return __half2float(__ushort_as_half((unsigned short)b)); }
template <> __device__ __forceinline__ float f16_bits<__nv_bfloat16>(unsigned int b) { return __uint_as_float(b << 16); }

// V values of a checkpoint field of element type UT, as floats
template <class UT, int V>
__device__ __forceinline__ void gldu(float (&d)[V], const UT* p)
{
    if constexpr (std::is_same<UT, float>::value) {
        gld<V>(d, p);
    } else {
        // two 16-bit values per 32-bit word, the lower address in the low half
        unsigned int w[V / 2];
        if constexpr (V == 4) {
            const uint2 t = __ldg(reinterpret_cast<const uint2*>(p));
            w[0] = t.x;
            w[1] = t.y;
        } else {
            w[0] = __ldg(reinterpret_cast<const unsigned int*>(p));
        }
#pragma unroll
        for (int k = 0; k < V / 2; ++k) {
            d[2 * k] = f16_bits<UT>(w[k] & 0xffffu);
            d[2 * k + 1] = f16_bits<UT>(w[k] >> 16);
        }
    }
}

template <int V>
__device__ __forceinline__ void sld(float (&d)[V], const float* p)
{
    if constexpr (V == 4) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        d[0] = t.x; d[1] = t.y; d[2] = t.z; d[3] = t.w;
    } else {
        const float2 t = *reinterpret_cast<const float2*>(p);
        d[0] = t.x; d[1] = t.y;
    }
}

template <int V>
__device__ __forceinline__ void vst(float* p, const float (&d)[V])
{
    if constexpr (V == 4) *reinterpret_cast<float4*>(p) = make_float4(d[0], d[1], d[2], d[3]);
    else *reinterpret_cast<float2*>(p) = make_float2(d[0], d[1]);
}

template <int V>
__device__ __forceinline__ void vstp(float* p, const float* d)
{
    if constexpr (V == 4) *reinterpret_cast<float4*>(p) = make_float4(d[0], d[1], d[2], d[3]);
    else *reinterpret_cast<float2*>(p) = make_float2(d[0], d[1]);
}

template <int V>
__device__ __forceinline__ void vzero(float (&d)[V])
{
#pragma unroll
    for (int i = 0; i < V; ++i) d[i] = 0.0f;
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Laplacian of the thread's V points (difference form, lap_at's order):
// z neighbours from the register queue (q[i] holds plane z - K + i), x and
// y neighbours from the staged plane.  Odd x offsets are formed per point:
// their operand pairs straddle register pairs, where two scalar additions
// cost less than building the packed operands.
template <int K, int V, int TX, int TY>
__device__ __forceinline__ void lap3(float (&out)[V], const float (&q)[2 * K + 1][V], const float* sm, int tx,
                                     int ty, const float* c)
{
    using G = G3<K, V, TX, TY>;
    const int r = ty + K;
    float xw[V + 2 * G::PX];
#pragma unroll
    for (int k = 0; k < G::NW; ++k) {
        float t[V];
        sld<V>(t, sm + r * G::RX + V * tx + V * k);
#pragma unroll
        for (int i = 0; i < V; ++i) xw[V * k + i] = t[i];
    }
    const float* u = q[K];
    float2 nu[V / 2], acc[V / 2];
#pragma unroll
    for (int p = 0; p < V / 2; ++p) {
        nu[p] = f2(-u[2 * p], -u[2 * p + 1]);
        acc[p] = f2(0.0f, 0.0f);
    }
#pragma unroll
    for (int j = K; j >= 1; --j) {
        float yp[V], ym[V];
        sld<V>(yp, sm + (r + j) * G::RX + G::PX + V * tx);
        sld<V>(ym, sm + (r - j) * G::RX + G::PX + V * tx);
        const float* zp = q[K + j];
        const float* zm = q[K - j];
        const float2 cj = f2(c[j], c[j]);
#pragma unroll
        for (int p = 0; p < V / 2; ++p) {
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
            acc[p] = __ffma2_rn(cj, s, acc[p]);
        }
    }
#pragma unroll
    for (int p = 0; p < V / 2; ++p) {
        out[2 * p] = acc[p].x;
        out[2 * p + 1] = acc[p].y;
    }
}

// leapfrog() for a pair of points (increment form, each lane rounding like
// the scalar operations): c + ((1 - e)(c - p) + w s) / (1 + e), e = eta dt/2
__device__ __forceinline__ float2 leap2v(float2 c, float2 p, float2 w, float2 s, float2 eta, float hdt)
{
    const float2 be = __ffma2_rn(f2(-eta.x, -eta.y), f2(hdt, hdt), f2(1.0f, 1.0f));
    const float2 d = __ffma2_rn(p, f2(-1.0f, -1.0f), c);                   // c - p, rounded once
    float2 t = __ffma2_rn(w, s, __fmul2_rn(be, d));
    t.x = eta.x != 0.0f ? __fdividef(t.x, __fmaf_rn(eta.x, hdt, 1.0f)) : t.x;
    t.y = eta.y != 0.0f ? __fdividef(t.y, __fmaf_rn(eta.y, hdt, 1.0f)) : t.y;
    return __fadd2_rn(c, t);
}

// Store V values into a 16-bit checkpoint field (BF16 or FP16): one V-wide
// store of packed values when the whole vector lies in the grid, else one
// value at a time.  Returns whether an FP16 value overflowed to infinity.
template <class T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ unsigned short bits16(__half h) { return __half_as_ushort(h); }
__device__ __forceinline__ unsigned short bits16(__nv_bfloat16 h) { return __bfloat16_as_ushort(h); }
__device__ __forceinline__ bool is_inf16(__half h) { return __hisinf(h) != 0; }
__device__ __forceinline__ bool is_inf16(__nv_bfloat16) { return false; }

template <class T, int V>
__device__ __forceinline__ bool st16(void* base, long long o, const float* v, bool full, int x0, int nx)
{
    T h[V];
    bool inf = false;
#pragma unroll
    for (int i = 0; i < V; ++i) {
        h[i] = from_f<T>(v[i]);
        inf = inf || ((full || x0 + i < nx) && is_inf16(h[i]));
    }
    T* p = static_cast<T*>(base) + o;
    if (full) {
        unsigned int w[V / 2];
#pragma unroll
        for (int k = 0; k < V / 2; ++k) w[k] = (unsigned int)bits16(h[2 * k]) | ((unsigned int)bits16(h[2 * k + 1]) << 16);
        if constexpr (V == 4) *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
        else *reinterpret_cast<unsigned int*>(p) = w[0];
    } else {
#pragma unroll
        for (int i = 0; i < V; ++i)
            if (x0 + i < nx) p[i] = h[i];
    }
    return inf;
}

template <int V>
struct Inj3 {                 // injection test of a thread's V points
    InjCol c0;                // the first point's column; point i is c0.base + i
    bool any;                 // some point's column meets the box
    int x0, nx;
    bool rowact;
    __device__ __forceinline__ void init(const Inj& in, int y, int x0_, int nx_, bool rowact_)
    {
        x0 = x0_;
        nx = nx_;
        rowact = rowact_;
        c0 = inj_col(in, y, x0, rowact);
        const int xe = min(x0 + V, nx);   // one past the last grid point of the vector
        any = in.on && rowact && y >= in.y0 && y < in.y1 && x0 < in.x1 && xe > in.x0;
    }
    __device__ __forceinline__ void add(float (&s)[V], const Inj& in, int z) const
    {
        if (any && z >= in.z0 && z < in.z1) {
#pragma unroll
            for (int i = 0; i < V; ++i) {
                InjCol c = c0;
                c.base += i;
                c.col = rowact && x0 + i < nx && x0 + i >= in.x0 && x0 + i < in.x1;
                s[i] = __fadd_rn(s[i], inj_val(in, c, z));
            }
        }
    }
};

// Where a thread's halo values of a plane come from (element offsets from
// the plane's origin-based row of the thread), and whether they exist.
template <int K, int V, int TX, int TY>
struct HaloMap {
    using G = G3<K, V, TX, TY>;
    int xo;            // first x-halo column: xb - PX (left) or xb + BXP (right), plus y * px
    int xs;            // staged offset of the x halo in the tile
    int ylo, yro;      // y halo rows: offsets of rows y - K and y + TY at column x0
    bool hx, hyl, hyr; // the x halo / y halo rows are loaded
    bool sx, sy;       // the thread stages x / y halo values
    __device__ __forceinline__ void init(int tx, int ty, int xb, int x0, int y, int nx, int ny, int px)
    {
        const int row = y * px;
        sx = tx == 0 || tx == TX - 1;
        sy = ty < K;
        if (tx == 0) {
            xo = row + xb - G::PX;
            xs = (ty + K) * G::RX;
            hx = y < ny;
        } else {
            xo = row + xb + G::BXP;
            xs = (ty + K) * G::RX + G::PX + G::BXP;
            hx = tx == TX - 1 && y < ny && xb + G::BXP < nx + K;
        }
        ylo = row - K * px + x0;
        yro = row + TY * px + x0;
        hyl = sy && x0 < nx;
        hyr = hyl && y + TY < ny + K;
    }
};

template <int K, int V, int TX, int TY>
struct HaloVals {
    using G = G3<K, V, TX, TY>;
    float xh[G::PX];
    float yl[V], yr[V];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int i = 0; i < G::PX; ++i) xh[i] = 0.0f;
        vzero<V>(yl);
        vzero<V>(yr);
    }
    // load the halo values of the plane whose origin-based offset is zoff
    template <class T>
    __device__ __forceinline__ void load(const T* __restrict__ f, int zoff, const HaloMap<K, V, TX, TY>& hm)
    {
        if (hm.hx) {
#pragma unroll
            for (int c = 0; c < G::PX; c += V) {
                float t[V];
                gldu<T, V>(t, f + zoff + hm.xo + c);
#pragma unroll
                for (int i = 0; i < V; ++i) xh[c + i] = t[i];
            }
        }
        if (hm.hyl) gldu<T, V>(yl, f + zoff + hm.ylo);
        if (hm.hyr) gldu<T, V>(yr, f + zoff + hm.yro);
    }
    // stage a plane: the thread's own values and its halo values
    __device__ __forceinline__ void store(float* sm, const float (&c)[V], int tx, int ty,
                                          const HaloMap<K, V, TX, TY>& hm) const
    {
        vst<V>(sm + (ty + K) * G::RX + G::PX + V * tx, c);
        if (hm.sx) {
#pragma unroll
            for (int i = 0; i < G::PX; i += V) {
                float t[V];
#pragma unroll
                for (int k = 0; k < V; ++k) t[k] = xh[i + k];
                vst<V>(sm + hm.xs + i, t);
            }
        }
        if (hm.sy) {
            vst<V>(sm + ty * G::RX + G::PX + V * tx, yl);
            vst<V>(sm + (ty + TY + K) * G::RX + G::PX + V * tx, yr);
        }
    }
};

// ------------------------------------------------------------- forward
// Step z: prefetch plane z+K+1 of u, u^{n-1} and w of plane z+1 and the
// halo values of plane z+1 (clamped at the end of the run, so the loads are
// unconditional and valid); barrier; compute plane z from the buffer staged
// in the previous step; stage plane z+1 into the other buffer.  Offsets are
// 32-bit element counts (the launcher checks the range).
template <int K, int V, int TX, int TY, int CK>
__device__ __forceinline__ void fwd3_body(const FwdArgs& a, float* smem, int bxi, int byi, int bzi, int gxn,
                                          int gyn)
{
    using G = G3<K, V, TX, TY>;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nz = a.g.nz, ny = a.g.ny, nx = a.g.nx;
    const int px = (int)a.g.px, pxy = (int)a.g.pxy;
    const int xb = bxi * G::BXP;
    const int x0 = xb + V * tx;
    const int y = byi * TY + ty;

    if (a.smp.n > 0) {   // receiver sampling of u^n by the first threads of the grid
        const int gt = ((bzi * gyn + byi) * gxn + bxi) * (TX * TY) + ty * TX + tx;
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
    const bool cload = rowact && x0 < nx;           // the thread's vector holds grid points
    const bool full = rowact && x0 + V <= nx;       // all V points are grid points
    const int col = y * px + x0;
    float ecol[V];
#pragma unroll
    for (int i = 0; i < V; ++i)
        ecol[i] = (rowact && x0 + i < nx) ? __fadd_rn(a.eta[nz + y], a.eta[nz + ny + x0 + i]) : 0.0f;
    Inj3<V> ij;
    ij.init(a.src, y, x0, nx, rowact);
    HaloMap<K, V, TX, TY> hm;
    hm.init(tx, ty, xb, x0, y, nx, ny, px);
    const float* __restrict__ U = a.u + col;
    const float* __restrict__ UP = a.up + col;
    const float* __restrict__ W = a.w + col;

    float q[2 * K + 1][V];
    float nq[V], nup[V], nw[V];
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) {
        if (cload) gld<V>(q[i], U + (z0 - K + i) * pxy);
        else vzero<V>(q[i]);
    }
    if (cload) {
        gld<V>(nq, U + (z0 + K) * pxy);
        gld<V>(nup, UP + z0 * pxy);
        gld<V>(nw, W + z0 * pxy);
    } else {
        vzero<V>(nq);
        vzero<V>(nup);
        vzero<V>(nw);
    }
    HaloVals<K, V, TX, TY> hv;
    hv.zero();
    hv.load(a.u, z0 * pxy, hm);
    hv.store(smem, q[K], tx, ty, hm);

    const int zqmax = nz + K - 1;
    for (int z = z0; z < z1; ++z) {
        const int P = (z - z0) & 1;
        float* sm = smem + P * G::TILE;
        float upv[V], wv[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            q[2 * K][i] = nq[i];
            upv[i] = nup[i];
            wv[i] = nw[i];
        }
        // prefetch (clamped, so the last step reads valid planes it does not use)
        const int zn = min(z + 1, z1 - 1);
        if (cload) {
            gld<V>(nq, U + min(z + K + 1, zqmax) * pxy);
            gld<V>(nup, UP + zn * pxy);
            gld<V>(nw, W + zn * pxy);
        }
        hv.load(a.u, zn * pxy, hm);
        __syncthreads();
        if (cload) {
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
        // stage plane z + 1 (its centre is already in the queue)
        hv.store(smem + (P ^ 1) * G::TILE, q[K + 1], tx, ty, hm);
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) {
#pragma unroll
            for (int k = 0; k < V; ++k) q[i][k] = q[i + 1][k];
        }
    }
}

// ------------------------------------------------------------- reverse
// Same structure as the forward step, with two staged fields (lam^j and
// u^{j-1}) and three point fields (lam^{j+1}, w, gacc) prefetched one plane
// ahead.
template <int K, int V, int TX, int TY, class UT>
__device__ __forceinline__ void adj3_body(const AdjArgs& a, float* smem, int bxi, int byi, int bzi)
{
    using G = G3<K, V, TX, TY>;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nz = a.g.nz, ny = a.g.ny, nx = a.g.nx;
    const int px = (int)a.g.px, pxy = (int)a.g.pxy;
    const int xb = bxi * G::BXP;
    const int x0 = xb + V * tx;
    const int y = byi * TY + ty;
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
    HaloMap<K, V, TX, TY> hm;
    hm.init(tx, ty, xb, x0, y, nx, ny, px);
    const UT* uu = static_cast<const UT*>(a.u);
    const float* __restrict__ L1 = a.l1 + col;
    const UT* __restrict__ UU = uu + col;
    const float* __restrict__ L2 = a.l2 + col;
    const float* __restrict__ W = a.w + col;
    const float* __restrict__ GA = a.gacc + col;

    float ql[2 * K + 1][V], qu[2 * K + 1][V];
    float nql[V], nqu[V], nl2[V], nw[V], ng[V];
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) {
        if (cload) {
            gld<V>(ql[i], L1 + (z0 - K + i) * pxy);
            gldu<UT, V>(qu[i], UU + (z0 - K + i) * pxy);
        } else {
            vzero<V>(ql[i]);
            vzero<V>(qu[i]);
        }
    }
    if (cload) {
        gld<V>(nql, L1 + (z0 + K) * pxy);
        gldu<UT, V>(nqu, UU + (z0 + K) * pxy);
        gld<V>(nl2, L2 + z0 * pxy);
        gld<V>(nw, W + z0 * pxy);
        gld_plain<V>(ng, GA + z0 * pxy);
    } else {
        vzero<V>(nql);
        vzero<V>(nqu);
        vzero<V>(nl2);
        vzero<V>(nw);
        vzero<V>(ng);
    }
    HaloVals<K, V, TX, TY> hl, hu;
    hl.zero();
    hu.zero();
    hl.load(a.l1, z0 * pxy, hm);
    hu.load(uu, z0 * pxy, hm);
    hl.store(smem, ql[K], tx, ty, hm);
    hu.store(smem + G::TILE, qu[K], tx, ty, hm);

    const int zqmax = nz + K - 1;
    for (int z = z0; z < z1; ++z) {
        const int P = (z - z0) & 1;
        float* sl = smem + P * (2 * G::TILE);
        float* su = sl + G::TILE;
        float l2v[V], wv[V], gv[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            ql[2 * K][i] = nql[i];
            qu[2 * K][i] = nqu[i];
            l2v[i] = nl2[i];
            wv[i] = nw[i];
            gv[i] = ng[i];
        }
        const int zn = min(z + 1, z1 - 1);
        if (cload) {
            const int zq = min(z + K + 1, zqmax) * pxy;
            gld<V>(nql, L1 + zq);
            gldu<UT, V>(nqu, UU + zq);
            gld<V>(nl2, L2 + zn * pxy);
            gld<V>(nw, W + zn * pxy);
            gld_plain<V>(ng, GA + zn * pxy);
        }
        hl.load(a.l1, zn * pxy, hm);
        hu.load(uu, zn * pxy, hm);
        __syncthreads();
        if (cload) {
            float sl_[V], su_[V];
            lap3<K, V, TX, TY>(sl_, ql, sl, tx, ty, a.c);
            ia.add(sl_, a.adj, z);
            lap3<K, V, TX, TY>(su_, qu, su, tx, ty, a.c);
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
        hl.store(smem + (P ^ 1) * (2 * G::TILE), ql[K + 1], tx, ty, hm);
        hu.store(smem + (P ^ 1) * (2 * G::TILE) + G::TILE, qu[K + 1], tx, ty, hm);
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) {
#pragma unroll
            for (int k = 0; k < V; ++k) {
                ql[i][k] = ql[i + 1][k];
                qu[i][k] = qu[i + 1][k];
            }
        }
    }
}

}  // namespace
}  // namespace ckfwi
