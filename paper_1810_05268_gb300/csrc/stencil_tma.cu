// TMA-fed 3D forward and reverse OT2 steps (space orders 2, 4, 8).
//
// Same arithmetic, in the same order, as kernels.cu (difference-form
// Laplacian, leapfrog with damping, CSR injections), so the results are
// bitwise those of the register-queue kernels; what changes is how data
// reaches the ALUs:
//   * a CTA owns a TX = 64 by TY block of (x, y) columns and a run of z
//     planes; every thread computes 4 consecutive x points;
//   * each halo'd (x, y) plane tile of a stencil field (TY + 2K rows of
//     TX + 2HX floats) arrives by one cp.async.bulk.tensor into a ring of
//     2K + 2 planes in shared memory, completion signalled on one mbarrier
//     per ring slot; the z neighbours are read from the ring, so there is
//     no per-thread halo staging, no register-queue shift and one CTA
//     barrier per plane (to release a slot before it is refilled);
//   * point fields (u^{n-1}, w, lam^{j+1}, g) are read with 128-bit loads
//     issued one plane ahead;
//   * arithmetic on point pairs uses the packed FP32x2 instructions
//     (__fadd2_rn, __ffma2_rn), which round each lane exactly like the
//     scalar ones.
// Waits on the mbarriers are bounded; a wait that runs out raises error bit
// 8 in a.err, the CTA stops at the next plane boundary and waits (bounded)
// for the copies it issued before leaving.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "internal.h"

namespace ckfwi {
namespace {

constexpr int TX = 64;                 // x points per CTA
constexpr int NTX = TX / 4;            // threads along x
constexpr int PF_FWD = 2;              // ring planes in flight beyond the stencil window
constexpr int PF_ADJ = 2;
constexpr long long WAIT_ROUNDS = 1LL << 22;

template <int K, int PF> struct RingCfg {
    static constexpr int HX = K <= 4 ? 4 : 8;            // x halo (multiple of 4 for TMA alignment)
    static constexpr int SXP = TX + 2 * HX;              // ring row pitch [elements]
    static constexpr int NS = 2 * K + 1 + PF;            // ring depth [planes]
};

__device__ __forceinline__ unsigned sm_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void column_of(int colidx, int ncx, int ty_, int* x0, int* y0)
{
    *x0 = (colidx % ncx) * TX;
    *y0 = (colidx / ncx) * ty_;
}

// first 128-byte aligned address of the dynamic shared memory (TMA
// destinations need it; the launch reserves 128 bytes of slack for this)
__device__ __forceinline__ unsigned char* align128(unsigned char* p)
{
    const unsigned a = sm_addr(p);
    return p + ((128u - (a & 127u)) & 127u);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sm_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(sm_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait with a short back-off, so that waiting warps yield their
// issue slots instead of spinning; `rounds` < 0 gives up without looking
// (how a test makes a wait run out without delaying any copy)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long rounds = WAIT_ROUNDS)
{
    if (rounds < 0) return false;
    for (int i = 0; i < 8; ++i)
        if (mbar_try(bar, parity)) return true;
    for (long long i = 0; i < rounds; ++i) {
        __nanosleep(32);
        if (mbar_try(bar, parity)) return true;
    }
    return false;
}

__device__ __forceinline__ void tma3(void* dst, const CUtensorMap* tm, int x, int y, int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(sm_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(z), "r"(sm_addr(bar))
        : "memory");
}

// 4 consecutive ring values as floats
template <class T> __device__ __forceinline__ float4 ld4(const T* p);
template <> __device__ __forceinline__ float4 ld4<float>(const float* p) { return *reinterpret_cast<const float4*>(p); }
template <> __device__ __forceinline__ float4 ld4<__nv_bfloat16>(const __nv_bfloat16* p)
{
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
template <> __device__ __forceinline__ float4 ld4<__half>(const __half* p)
{
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ float2 lo(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 sum_of_diffs(float2 a, float2 b, float2 nu)
{
    return __fadd2_rn(__fadd2_rn(a, nu), __fadd2_rn(b, nu));          // (a - u) + (b - u)
}

// Ring of planes of one stencil field; the TMA box is (SXP, TY + 2K, 1).
template <int K, int TY, class T, int PF>
struct Ring {
    static constexpr int SXP = RingCfg<K, PF>::SXP;
    static constexpr int NS = RingCfg<K, PF>::NS;
    static constexpr int PLANE = (TY + 2 * K) * SXP;                 // elements of one plane tile
    static constexpr unsigned BYTES = PLANE * sizeof(T);             // bytes a TMA copy delivers
    static constexpr unsigned STRIDE = (BYTES + 127) / 128 * 128;    // plane stride (128-B aligned)
    T* buf;
    uint64_t* bar;
    __device__ __forceinline__ const T* plane(int slot) const
    {
        return reinterpret_cast<const T*>(reinterpret_cast<const unsigned char*>(buf) + slot * STRIDE);
    }
    __device__ __forceinline__ T* plane_w(int slot) const
    {
        return reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(buf) + slot * STRIDE);
    }
};

// Shared-memory views of the rings in units of 4 elements (16 bytes for
// float, 8 bytes for the 16-bit types); a window entry is the index of this
// thread's 4 points in one plane, so every load below is [index + constant].
extern __shared__ __align__(128) unsigned char smem_raw[];

template <class T> struct G4;
template <> struct G4<float> {
    __device__ __forceinline__ static float4 at(unsigned byte_base, int i)
    {
        return reinterpret_cast<const float4*>(smem_raw + byte_base)[i];
    }
};
template <> struct G4<__nv_bfloat16> {
    __device__ __forceinline__ static float4 at(unsigned byte_base, int i)
    {
        const uint2 v = reinterpret_cast<const uint2*>(smem_raw + byte_base)[i];
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
};
template <> struct G4<__half> {
    __device__ __forceinline__ static float4 at(unsigned byte_base, int i)
    {
        const uint2 v = reinterpret_cast<const uint2*>(smem_raw + byte_base)[i];
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
};

__device__ __forceinline__ float xdiff(float p, float m, float u) { return __fadd_rn(__fsub_rn(p, u), __fsub_rn(m, u)); }

// Difference-form Laplacian of 4 x-consecutive points (see kernels.cu),
// summed over j = K..1 in the order z, x, y.  q[d]: index of the thread's
// 4 points in the plane of offset d - K (ring relative to byte_base).
template <int K, class T>
__device__ __forceinline__ void lap4(unsigned byte_base, const int* q, const float* cj, float4& centre, float2& acc0,
                                     float2& acc1)
{
    constexpr int HX = K <= 4 ? 4 : 8;
    constexpr int ROW = (TX + 2 * HX) / 4;          // ring row pitch in groups of 4
    float xv[4 + 2 * HX];
#pragma unroll
    for (int m = 0; m < (4 + 2 * HX) / 4; ++m) {
        const float4 t = G4<T>::at(byte_base, q[K] - HX / 4 + m);
        xv[4 * m] = t.x; xv[4 * m + 1] = t.y; xv[4 * m + 2] = t.z; xv[4 * m + 3] = t.w;
    }
    centre = make_float4(xv[HX], xv[HX + 1], xv[HX + 2], xv[HX + 3]);
    const float2 nu0 = make_float2(-centre.x, -centre.y), nu1 = make_float2(-centre.z, -centre.w);
    acc0 = make_float2(0.0f, 0.0f);
    acc1 = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int j = K; j >= 1; --j) {
        const float4 zp = G4<T>::at(byte_base, q[K + j]);
        const float4 zm = G4<T>::at(byte_base, q[K - j]);
        const float4 yp = G4<T>::at(byte_base, q[K] + j * ROW);
        const float4 ym = G4<T>::at(byte_base, q[K] - j * ROW);
        float2 s0 = sum_of_diffs(lo(zp), lo(zm), nu0);
        float2 s1 = sum_of_diffs(hi(zp), hi(zm), nu1);
        const float2 x0 = make_float2(xdiff(xv[HX + j], xv[HX - j], centre.x), xdiff(xv[HX + 1 + j], xv[HX + 1 - j], centre.y));
        const float2 x1 = make_float2(xdiff(xv[HX + 2 + j], xv[HX + 2 - j], centre.z), xdiff(xv[HX + 3 + j], xv[HX + 3 - j], centre.w));
        s0 = __fadd2_rn(s0, x0);
        s1 = __fadd2_rn(s1, x1);
        s0 = __fadd2_rn(s0, sum_of_diffs(lo(yp), lo(ym), nu0));
        s1 = __fadd2_rn(s1, sum_of_diffs(hi(yp), hi(ym), nu1));
        const float2 c2 = make_float2(cj[j], cj[j]);
        acc0 = __ffma2_rn(c2, s0, acc0);
        acc1 = __ffma2_rn(c2, s1, acc1);
    }
}

// Per-thread part of a CSR injection for 4 x-consecutive points.
struct Inj4 {
    int mask;            // bit i: point i inside the box's (y, x) range
    int base;            // box-local index of point 0's column in a plane
    int plane;
};

__device__ __forceinline__ Inj4 inj4(const Inj& in, int y, int x, int nx, bool row)
{
    Inj4 c{0, 0, 0};
    if (!in.on || !row || y < in.y0 || y >= in.y1) return c;
    c.plane = (in.y1 - in.y0) * (in.x1 - in.x0);
    c.base = (y - in.y0) * (in.x1 - in.x0) + (x - in.x0);
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (x + i < nx && x + i >= in.x0 && x + i < in.x1) c.mask |= 1 << i;
    return c;
}

__device__ __forceinline__ float inj1(const Inj& in, int b)
{
    float acc = 0.0f;
    const int e1 = in.rowptr[b + 1];
    for (int e = in.rowptr[b]; e < e1; ++e) acc = __fmaf_rn(in.wt[e], in.series[in.col[e]], acc);
    return acc;
}

__device__ __forceinline__ float4 inj_vals(const Inj& in, const Inj4& c, int z)
{
    float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (c.mask && z >= in.z0 && z < in.z1) {
        const int b = (z - in.z0) * c.plane + c.base;
        if (c.mask & 1) v.x = inj1(in, b);
        if (c.mask & 2) v.y = inj1(in, b + 1);
        if (c.mask & 4) v.z = inj1(in, b + 2);
        if (c.mask & 8) v.w = inj1(in, b + 3);
    }
    return v;
}

// leapfrog() of a point pair (increment form, each lane rounding like the
// scalar operations): c + ((1 - e)(c - p) + w s) / (1 + e), e = eta dt/2
__device__ __forceinline__ float2 leap2(float2 c, float2 p, float2 w, float2 s, float2 eta, float hdt)
{
    const float2 be = make_float2(__fmaf_rn(-eta.x, hdt, 1.0f), __fmaf_rn(-eta.y, hdt, 1.0f));
    const float2 d = __ffma2_rn(p, make_float2(-1.0f, -1.0f), c);          // c - p, rounded once
    float2 t = __ffma2_rn(w, s, __fmul2_rn(be, d));
    t.x = eta.x != 0.0f ? __fdividef(t.x, __fmaf_rn(eta.x, hdt, 1.0f)) : t.x;
    t.y = eta.y != 0.0f ? __fdividef(t.y, __fmaf_rn(eta.y, hdt, 1.0f)) : t.y;
    return __fadd2_rn(c, t);
}

__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

// store 4 points (all, or the ones below nx)
__device__ __forceinline__ void st4(float* p, const float4& v, int nvalid)
{
    if (nvalid >= 4) {
        *reinterpret_cast<float4*>(p) = v;
    } else {
        if (nvalid > 0) p[0] = v.x;
        if (nvalid > 1) p[1] = v.y;
        if (nvalid > 2) p[2] = v.z;
    }
}

template <class H2, class H, class CV>
__device__ __forceinline__ void st4h(H* p, const float4& v, int nvalid, CV cvt)
{
    const H a = cvt(v.x), b = cvt(v.y), c = cvt(v.z), d = cvt(v.w);
    if (nvalid >= 4) {
        H2 lo2, hi2;
        lo2.x = a; lo2.y = b;
        hi2.x = c; hi2.y = d;
        uint2 u;
        u.x = *reinterpret_cast<unsigned*>(&lo2);
        u.y = *reinterpret_cast<unsigned*>(&hi2);
        *reinterpret_cast<uint2*>(p) = u;
    } else {
        if (nvalid > 0) p[0] = a;
        if (nvalid > 1) p[1] = b;
        if (nvalid > 2) p[2] = c;
    }
}

// A CTA numbers the planes it loads 0, 1, 2, ... across all its column
// segments (kb = number of planes of earlier segments); plane number k sits
// in ring slot k % NS and completes phase (k / NS) of that slot's barrier.
template <int K, int TY, class T, int PF>
__device__ __forceinline__ void ring_init(Ring<K, TY, T, PF>& R, int tid)
{
    if (tid == 0) {
        for (int s = 0; s < Ring<K, TY, T, PF>::NS; ++s) mbar_init(&R.bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
}

template <int K, int TY, class T, int PF>
__device__ __forceinline__ void ring_issue(Ring<K, TY, T, PF>& R, const CUtensorMap* tm, int x0, int y0, int zz, int zb,
                                           int kb, int H)
{
    constexpr int NS = Ring<K, TY, T, PF>::NS;
    const int k = kb + (zz - zb);
    const int s = k % NS;
    // The slot's previous plane was only read (into registers) by the CTA,
    // and every thread passed the CTA barrier after those reads, so the
    // copy may overwrite it without a proxy fence (one is needed only when
    // generic-proxy writes to shared memory are to be read by the async proxy).
    mbar_expect_tx(&R.bar[s], Ring<K, TY, T, PF>::BYTES);
    tma3(R.plane_w(s), tm, x0, y0, zz + H, &R.bar[s]);
}

// first window of a segment: planes zb .. min(zlast, zb + NS - 1)
template <int K, int TY, class T, int PF>
__device__ __forceinline__ void ring_prologue(Ring<K, TY, T, PF>& R, const CUtensorMap* tm, int x0, int y0, int zb,
                                              int zlast, int kb, int H, int tid)
{
    if (tid == 0)
        for (int zz = zb; zz <= zlast && zz < zb + Ring<K, TY, T, PF>::NS; ++zz) ring_issue(R, tm, x0, y0, zz, zb, kb, H);
}

template <int K, int TY, class T, int PF>
__device__ __forceinline__ bool ring_wait(const Ring<K, TY, T, PF>& R, int zz, int zb, int kb,
                                          long long rounds = WAIT_ROUNDS)
{
    constexpr int NS = Ring<K, TY, T, PF>::NS;
    const int k = kb + (zz - zb);
    return mbar_wait(&R.bar[k % NS], (unsigned)((k / NS) & 1), rounds);
}

// After the CTA barrier of plane z: the slot of plane z-K takes plane z-K+NS.
template <int K, int TY, class T, int PF>
__device__ __forceinline__ void ring_refill(Ring<K, TY, T, PF>& R, const CUtensorMap* tm, int x0, int y0, int z, int zb,
                                            int zlast, int kb, int H)
{
    constexpr int NS = Ring<K, TY, T, PF>::NS;
    const int zn = z - K + NS;
    if (zn <= zlast) ring_issue(R, tm, x0, y0, zn, zb, kb, H);
}

// On an aborted run: wait (bounded, always the full WAIT_ROUNDS) for every
// plane still held or in flight (planes max(zb, z-K) .. the last one
// issued), so that no copy lands in shared memory after the CTA has left.
template <int K, int TY, class T, int PF>
__device__ __forceinline__ void ring_drain(const Ring<K, TY, T, PF>& R, int z, int zb, int zlast, int kb)
{
    constexpr int NS = Ring<K, TY, T, PF>::NS;
    const int hi_issued = min(zlast, z - K + NS - 1);
    for (int zz = max(zb, z - K); zz <= hi_issued; ++zz) ring_wait(R, zz, zb, kb);
}

// Group indices of the stencil window z-K .. z+K, rotated by one slot per plane.
template <int K, int TY, class T, int PF>
struct Window {
    int q[2 * K + 1];
    int next;            // ring slot of plane z+K+1
    int off;             // this thread's group index inside a plane
    static constexpr int PG = Ring<K, TY, T, PF>::STRIDE / (4 * sizeof(T));   // groups per plane slot
    __device__ __forceinline__ void init(int kb, int r, int c)
    {
        constexpr int NS = Ring<K, TY, T, PF>::NS;
        off = (r * Ring<K, TY, T, PF>::SXP + c) / 4;
#pragma unroll
        for (int d = 0; d <= 2 * K; ++d) q[d] = ((kb + d) % NS) * PG + off;
        next = (kb + 2 * K + 1) % NS;
    }
    __device__ __forceinline__ void advance()
    {
#pragma unroll
        for (int d = 0; d < 2 * K; ++d) q[d] = q[d + 1];
        q[2 * K] = next * PG + off;
        next = (next + 1 == Ring<K, TY, T, PF>::NS) ? 0 : next + 1;
    }
};

// Persistent work split: the (x, y) column tiles (x fastest) times the nz
// planes form W = ncols * nz units; CTA i of G takes units
// [i W / G, (i+1) W / G) in order, i.e. one or more z segments of one or two
// columns.  No wave quantisation, one pipeline fill per segment.
struct Work {
    long long w, wend;
    int ncx, nz;
    __device__ __forceinline__ void init(int ncols, int ncx_, int nz_)
    {
        ncx = ncx_;
        nz = nz_;
        const long long W = (long long)ncols * nz;
        w = W * blockIdx.x / gridDim.x;
        wend = W * (blockIdx.x + 1) / gridDim.x;
    }
    // next segment: column index and plane range [za, zc)
    __device__ __forceinline__ bool next(int* col, int* za, int* zc)
    {
        if (w >= wend) return false;
        *col = (int)(w / nz);
        *za = (int)(w % nz);
        *zc = (int)min((long long)nz, *za + (wend - w));
        w += *zc - *za;
        return true;
    }
};

template <int K, int TY, int CK>
__global__ void __launch_bounds__(NTX * TY) fwd_tma_kernel(const FwdArgs a, const __grid_constant__ CUtensorMap tmu)
{
    using RU = Ring<K, TY, float, PF_FWD>;
    __shared__ int abort_s[2];   // a wait gave up at a plane step of this parity
    unsigned char* smem = align128(smem_raw);
    const unsigned base_u = (unsigned)(smem - smem_raw);
    RU R{reinterpret_cast<float*>(smem), reinterpret_cast<uint64_t*>(smem + RU::NS * RU::STRIDE)};
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * NTX + tx;
    const int nz = a.g.nz, ny = a.g.ny, nx = a.g.nx, H = a.g.H;
    const long long px = a.g.px, pxy = a.g.pxy;

    if (a.smp.n > 0) {   // receiver sampling of u^n by the first threads of the grid
        const int gt = (int)blockIdx.x * (NTX * TY) + tid;
        for (int r = gt; r < a.smp.n; r += gridDim.x * NTX * TY) {
            float acc = 0.0f;
            for (int i = 0; i < a.smp.nst; ++i)
                acc = __fmaf_rn(a.smp.wt[r * a.smp.nst + i], __ldg(a.u + a.smp.idx[r * a.smp.nst + i]), acc);
            a.smp.out[r] = acc;
        }
    }
    const int ncx = (nx + TX - 1) / TX, ncy = (ny + TY - 1) / TY;
    Work wk;
    wk.init(ncx * ncy, ncx, nz);
    if (tid == 0) abort_s[0] = abort_s[1] = 0;
    ring_init(R, tid);
    __syncthreads();
    int kb = 0;
    int col, za, zc;
    bool ok = true;
    bool aborted = false;        // the same in every thread: read after one barrier
    int ph = 0;                  // parity of the plane steps so far
    while (wk.next(&col, &za, &zc)) {
        int x0, y0;
        column_of(col, ncx, TY, &x0, &y0);
        const int x = x0 + 4 * tx, y = y0 + ty;
        const bool row = y < ny;
        const bool act = row && x < nx;
        const int nvalid = act ? min(4, nx - x) : 0;
        const int zb = za - K, zlast = zc - 1 + K;
        ring_prologue(R, &tmu, x0, y0, zb, zlast, kb, H, tid);
        float4 ecol = make_float4(0.f, 0.f, 0.f, 0.f);
        if (act) {
            const float ey = a.eta[nz + y];
            const float* ex = a.eta + nz + ny + x;
            ecol.x = ey + ex[0];
            if (nvalid > 1) ecol.y = ey + ex[1];
            if (nvalid > 2) ecol.z = ey + ex[2];
            if (nvalid > 3) ecol.w = ey + ex[3];
        }
        const Inj4 ic = inj4(a.src, y, x, nx, row);
        const int r = ty + K, c = RingCfg<K, PF_FWD>::HX + 4 * tx;
        for (int zz = zb; zz < za + K; ++zz) ok &= ring_wait(R, zz, zb, kb, a.wait_limit);
        Window<K, TY, float, PF_FWD> W;
        W.init(kb, r, c);
        const long long colo = (long long)y * px + x;
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 up0 = zero4, w0 = zero4, up1 = zero4, w1 = zero4;
        if (act) {
            up0 = ldg4(a.up + (long long)za * pxy + colo);
            w0 = ldg4(a.w + (long long)za * pxy + colo);
            if (za + 1 < zc) {
                up1 = ldg4(a.up + (long long)(za + 1) * pxy + colo);
                w1 = ldg4(a.w + (long long)(za + 1) * pxy + colo);
            }
        }
        int z = za;
        for (; z < zc; ++z) {
            ok &= ring_wait(R, z + K, zb, kb, a.wait_limit);
            const float4 upv = up0, wv = w0;
            up0 = up1;
            w0 = w1;
            if (act && z + 2 < zc) {
                up1 = ldg4(a.up + (long long)(z + 2) * pxy + colo);
                w1 = ldg4(a.w + (long long)(z + 2) * pxy + colo);
            }
            if (act && ok) {
                float4 u;
                float2 l0, l1;
                lap4<K, float>(base_u, W.q, a.c, u, l0, l1);
                const float4 q = inj_vals(a.src, ic, z);
                l0 = __fadd2_rn(l0, lo(q));
                l1 = __fadd2_rn(l1, hi(q));
                const float ez = a.eta[z];
                const float2 e0 = make_float2(ez + ecol.x, ez + ecol.y), e1 = make_float2(ez + ecol.z, ez + ecol.w);
                const float2 v0 = leap2(lo(u), lo(upv), lo(wv), l0, e0, a.hdt);
                const float2 v1 = leap2(hi(u), hi(upv), hi(wv), l1, e1, a.hdt);
                const float4 v = make_float4(v0.x, v0.y, v1.x, v1.y);
                const long long o = (long long)z * pxy + colo;
                st4(a.out + o, v, nvalid);
                if (CK == CK_FP32) {
                    st4(static_cast<float*>(a.ck_up) + o, u, nvalid);
                } else if (CK == CK_BF16) {
                    auto cv = [](float f) { return __float2bfloat16_rn(f); };
                    st4h<__nv_bfloat162>(static_cast<__nv_bfloat16*>(a.ck_u) + o, v, nvalid, cv);
                    st4h<__nv_bfloat162>(static_cast<__nv_bfloat16*>(a.ck_up) + o, u, nvalid, cv);
                } else if (CK == CK_FP16) {
                    auto cv = [](float f) { return __float2half_rn(f); };
                    st4h<__half2>(static_cast<__half*>(a.ck_u) + o, v, nvalid, cv);
                    st4h<__half2>(static_cast<__half*>(a.ck_up) + o, u, nvalid, cv);
                    float mx = fmaxf(fabsf(v.x), fabsf(u.x));
                    if (nvalid > 1) mx = fmaxf(mx, fmaxf(fabsf(v.y), fabsf(u.y)));
                    if (nvalid > 2) mx = fmaxf(mx, fmaxf(fabsf(v.z), fabsf(u.z)));
                    if (nvalid > 3) mx = fmaxf(mx, fmaxf(fabsf(v.w), fabsf(u.w)));
                    if (__hisinf(__float2half_rn(mx))) atomicOr(a.err, 1);
                }
            }
            // a thread one step ahead flags the other slot, so all threads
            // leave at the same plane
            if (!ok) abort_s[ph] = 1;
            __syncthreads();
            if (abort_s[ph]) {
                aborted = true;
                break;
            }
            ph ^= 1;
            if (tid == 0) ring_refill(R, &tmu, x0, y0, z, zb, zlast, kb, H);
            W.advance();
        }
        if (aborted) {
            if (tid == 0) {
                atomicOr(a.err, 8);
                ring_drain(R, z, zb, zlast, kb);
            }
            return;
        }
        kb += zlast - zb + 1;
    }
}

template <int K, int TY, class UT>
__global__ void __launch_bounds__(NTX * TY) adj_tma_kernel(const AdjArgs a, const __grid_constant__ CUtensorMap tml,
                                                           const __grid_constant__ CUtensorMap tmu)
{
    using RL = Ring<K, TY, float, PF_ADJ>;
    using RUu = Ring<K, TY, UT, PF_ADJ>;
    __shared__ int abort_s[2];
    unsigned char* smem = align128(smem_raw);
    const unsigned base_l = (unsigned)(smem - smem_raw);
    const unsigned base_uu = base_l + RL::NS * RL::STRIDE;
    RL L{reinterpret_cast<float*>(smem), reinterpret_cast<uint64_t*>(smem + RL::NS * RL::STRIDE + RUu::NS * RUu::STRIDE)};
    RUu U{reinterpret_cast<UT*>(smem + RL::NS * RL::STRIDE), L.bar + RL::NS};
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * NTX + tx;
    const int nz = a.g.nz, ny = a.g.ny, nx = a.g.nx, H = a.g.H;
    const long long px = a.g.px, pxy = a.g.pxy;
    const int ncx = (nx + TX - 1) / TX, ncy = (ny + TY - 1) / TY;
    Work wk;
    wk.init(ncx * ncy, ncx, nz);
    if (tid == 0) abort_s[0] = abort_s[1] = 0;
    ring_init(L, tid);
    ring_init(U, tid);
    __syncthreads();
    int kb = 0;
    int col, za, zc;
    bool ok = true;
    bool aborted = false;        // the same in every thread: read after one barrier
    int ph = 0;                  // parity of the plane steps so far
    while (wk.next(&col, &za, &zc)) {
        int x0, y0;
        column_of(col, ncx, TY, &x0, &y0);
        const int x = x0 + 4 * tx, y = y0 + ty;
        const bool row = y < ny;
        const bool act = row && x < nx;
        const int nvalid = act ? min(4, nx - x) : 0;
        const int zb = za - K, zlast = zc - 1 + K;
        ring_prologue(L, &tml, x0, y0, zb, zlast, kb, H, tid);
        ring_prologue(U, &tmu, x0, y0, zb, zlast, kb, H, tid);
        float4 ecol = make_float4(0.f, 0.f, 0.f, 0.f);
        if (act) {
            const float ey = a.eta[nz + y];
            const float* ex = a.eta + nz + ny + x;
            ecol.x = ey + ex[0];
            if (nvalid > 1) ecol.y = ey + ex[1];
            if (nvalid > 2) ecol.z = ey + ex[2];
            if (nvalid > 3) ecol.w = ey + ex[3];
        }
        const Inj4 ia = inj4(a.adj, y, x, nx, row);
        const Inj4 is = inj4(a.src, y, x, nx, row);
        const int r = ty + K, c = RingCfg<K, PF_ADJ>::HX + 4 * tx;
        for (int zz = zb; zz < za + K; ++zz) {
            ok &= ring_wait(L, zz, zb, kb, a.wait_limit);
            ok &= ring_wait(U, zz, zb, kb, a.wait_limit);
        }
        Window<K, TY, float, PF_ADJ> WL;
        Window<K, TY, UT, PF_ADJ> WU;
        WL.init(kb, r, c);
        WU.init(kb, r, c);
        const long long colo = (long long)y * px + x;
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 l20 = zero4, w0 = zero4, g0v = zero4, l21 = zero4, w1 = zero4, g1v = zero4;
        if (act) {
            const long long o0 = (long long)za * pxy + colo;
            l20 = ldg4(a.l2 + o0);
            w0 = ldg4(a.w + o0);
            g0v = *reinterpret_cast<const float4*>(a.gacc + o0);
            if (za + 1 < zc) {
                l21 = ldg4(a.l2 + o0 + pxy);
                w1 = ldg4(a.w + o0 + pxy);
                g1v = *reinterpret_cast<const float4*>(a.gacc + o0 + pxy);
            }
        }
        int z = za;
        for (; z < zc; ++z) {
            ok &= ring_wait(L, z + K, zb, kb, a.wait_limit);
            ok &= ring_wait(U, z + K, zb, kb, a.wait_limit);
            const float4 l2v = l20, wv = w0, gv = g0v;
            l20 = l21;
            w0 = w1;
            g0v = g1v;
            if (act && z + 2 < zc) {
                const long long o2 = (long long)(z + 2) * pxy + colo;
                l21 = ldg4(a.l2 + o2);
                w1 = ldg4(a.w + o2);
                g1v = *reinterpret_cast<const float4*>(a.gacc + o2);
            }
            if (act && ok) {
                float4 lc, uc;
                float2 a0, a1, b0, b1;
                lap4<K, float>(base_l, WL.q, a.c, lc, a0, a1);
                const float4 qa = inj_vals(a.adj, ia, z);
                a0 = __fadd2_rn(a0, lo(qa));
                a1 = __fadd2_rn(a1, hi(qa));
                lap4<K, UT>(base_uu, WU.q, a.c, uc, b0, b1);
                const float4 qs = inj_vals(a.src, is, z);
                b0 = __fadd2_rn(b0, lo(qs));
                b1 = __fadd2_rn(b1, hi(qs));
                const float ez = a.eta[z];
                const float2 e0 = make_float2(ez + ecol.x, ez + ecol.y), e1 = make_float2(ez + ecol.z, ez + ecol.w);
                const float2 v0 = leap2(lo(lc), lo(l2v), lo(wv), a0, e0, a.hdt);
                const float2 v1 = leap2(hi(lc), hi(l2v), hi(wv), a1, e1, a.hdt);
                const float2 g0 = __ffma2_rn(v0, b0, lo(gv));
                const float2 g1 = __ffma2_rn(v1, b1, hi(gv));
                const long long o = (long long)z * pxy + colo;
                st4(a.l0 + o, make_float4(v0.x, v0.y, v1.x, v1.y), nvalid);
                st4(a.gacc + o, make_float4(g0.x, g0.y, g1.x, g1.y), nvalid);
            }
            // a thread one step ahead flags the other slot, so all threads
            // leave at the same plane
            if (!ok) abort_s[ph] = 1;
            __syncthreads();
            if (abort_s[ph]) {
                aborted = true;
                break;
            }
            ph ^= 1;
            if (tid == 0) {
                ring_refill(L, &tml, x0, y0, z, zb, zlast, kb, H);
                ring_refill(U, &tmu, x0, y0, z, zb, zlast, kb, H);
            }
            WL.advance();
            WU.advance();
        }
        if (aborted) {
            if (tid == 0) {
                atomicOr(a.err, 8);
                ring_drain(L, z, zb, zlast, kb);
                ring_drain(U, z, zb, zlast, kb);
            }
            return;
        }
        kb += zlast - zb + 1;
    }
}

template <int K, int TY>
size_t fwd_smem()
{
    using RU = Ring<K, TY, float, PF_FWD>;
    return 128 + (size_t)RU::NS * RU::STRIDE + RU::NS * sizeof(uint64_t);
}

template <int K, int TY, class UT>
size_t adj_smem()
{
    using RL = Ring<K, TY, float, PF_ADJ>;
    using RUu = Ring<K, TY, UT, PF_ADJ>;
    return 128 + (size_t)RL::NS * RL::STRIDE + RUu::NS * RUu::STRIDE + (RL::NS + RUu::NS) * sizeof(uint64_t);
}

template <class F>
cudaError_t prep(F kern, size_t sh)
{
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
}

int num_sms()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// persistent grid: zlen carries the CTAs per SM
dim3 tma_grid(const FieldGeom& g, int ty, int per_sm)
{
    const long long ncols = (long long)((g.nx + TX - 1) / TX) * ((g.ny + ty - 1) / ty);
    long long G = (long long)num_sms() * per_sm;
    G = std::min(G, ncols * g.nz);
    return dim3((unsigned)std::max<long long>(G, 1), 1, 1);
}

template <int K, int TY>
cudaError_t fwd_go(const FwdArgs& a, const CUtensorMap& tm, int ck, cudaStream_t s)
{
    const dim3 blk(NTX, TY, 1);
    const dim3 grd = tma_grid(a.g, TY, a.zlen);
    const size_t sh = fwd_smem<K, TY>();
    cudaError_t e = cudaSuccess;
    switch (ck) {
    case CK_NONE:
        if ((e = prep(fwd_tma_kernel<K, TY, CK_NONE>, sh)) == cudaSuccess) fwd_tma_kernel<K, TY, CK_NONE><<<grd, blk, sh, s>>>(a, tm);
        break;
    case CK_FP32:
        if ((e = prep(fwd_tma_kernel<K, TY, CK_FP32>, sh)) == cudaSuccess) fwd_tma_kernel<K, TY, CK_FP32><<<grd, blk, sh, s>>>(a, tm);
        break;
    case CK_BF16:
        if ((e = prep(fwd_tma_kernel<K, TY, CK_BF16>, sh)) == cudaSuccess) fwd_tma_kernel<K, TY, CK_BF16><<<grd, blk, sh, s>>>(a, tm);
        break;
    case CK_FP16:
        if ((e = prep(fwd_tma_kernel<K, TY, CK_FP16>, sh)) == cudaSuccess) fwd_tma_kernel<K, TY, CK_FP16><<<grd, blk, sh, s>>>(a, tm);
        break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int K, int TY>
cudaError_t adj_go(const AdjArgs& a, const CUtensorMap& tml, const CUtensorMap& tmu, int ut, cudaStream_t s)
{
    const dim3 blk(NTX, TY, 1);
    const dim3 grd = tma_grid(a.g, TY, a.zlen);
    cudaError_t e = cudaSuccess;
    switch (ut) {
    case U_FP32: {
        const size_t sh = adj_smem<K, TY, float>();
        if ((e = prep(adj_tma_kernel<K, TY, float>, sh)) == cudaSuccess) adj_tma_kernel<K, TY, float><<<grd, blk, sh, s>>>(a, tml, tmu);
        break;
    }
    case U_BF16: {
        const size_t sh = adj_smem<K, TY, __nv_bfloat16>();
        if ((e = prep(adj_tma_kernel<K, TY, __nv_bfloat16>, sh)) == cudaSuccess) adj_tma_kernel<K, TY, __nv_bfloat16><<<grd, blk, sh, s>>>(a, tml, tmu);
        break;
    }
    case U_FP16: {
        const size_t sh = adj_smem<K, TY, __half>();
        if ((e = prep(adj_tma_kernel<K, TY, __half>, sh)) == cudaSuccess) adj_tma_kernel<K, TY, __half><<<grd, blk, sh, s>>>(a, tml, tmu);
        break;
    }
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int K>
cudaError_t fwd_k(const FwdArgs& a, const CUtensorMap& tm, int ty, int ck, cudaStream_t s)
{
    if (ty == 8) return fwd_go<K, 8>(a, tm, ck, s);
    if (ty == 16) return fwd_go<K, 16>(a, tm, ck, s);
    return cudaErrorInvalidValue;
}

template <int K>
cudaError_t adj_k(const AdjArgs& a, const CUtensorMap& tml, const CUtensorMap& tmu, int ty, int ut, cudaStream_t s)
{
    if (ty == 8) return adj_go<K, 8>(a, tml, tmu, ut, s);
    if (ty == 16) return adj_go<K, 16>(a, tml, tmu, ut, s);
    return cudaErrorInvalidValue;
}

}  // namespace

int tma_halo_x(int K) { return K <= 4 ? 4 : 8; }
int tma_tile_x() { return TX; }

bool tma_supported(int dims, int K, int ty)
{
    return dims == 3 && (K == 1 || K == 2 || K == 4) && (ty == 8 || ty == 16);
}

cudaError_t launch_fwd_tma(const FwdArgs& a, const CUtensorMap& tmu, const Tile& t, int K, int ck, cudaStream_t s)
{
    FwdArgs b = a;
    b.zlen = t.zlen;
    switch (K) {
    case 1: return fwd_k<1>(b, tmu, t.by, ck, s);
    case 2: return fwd_k<2>(b, tmu, t.by, ck, s);
    case 4: return fwd_k<4>(b, tmu, t.by, ck, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adj_tma(const AdjArgs& a, const CUtensorMap& tml, const CUtensorMap& tmu, const Tile& t, int K,
                           int ut, cudaStream_t s)
{
    AdjArgs b = a;
    b.zlen = t.zlen;
    switch (K) {
    case 1: return adj_k<1>(b, tml, tmu, t.by, ut, s);
    case 2: return adj_k<2>(b, tml, tmu, t.by, ut, s);
    case 4: return adj_k<4>(b, tml, tmu, t.by, ut, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ckfwi
