// Stencil steps fed by tensor copies, with a register z queue (3D,
// Tile.ver 8): the forward step, and the reverse step split into its
// lambda half (the same forward kernel on the adjoint field with the
// adjoint injection) and its gradient half (gradq_kernel).
//
// The async-copy generation (stencil_v4.cu) has every thread issue its own
// copies of a plane: its vector of the u tile, at most one halo vector, its
// vectors of u^{n-1} and w, each with an address, a predicate and a
// zero-fill size, and keeps those copy descriptors in registers.  Here one
// thread issues three tensor copies a plane instead (cp.async.bulk.tensor):
// the halo'd tile of plane z + K + D of the staged field and the point
// tiles of plane z + D (D = 1 or 2 planes of prefetch, Tile.pf; 0 reads as
// 1), all completing on the mbarrier of their ring slot.  The other
// threads only wait on that barrier.  Everything else is the async-copy
// generation's: a 32 x 16 tile, four x points a thread, the queue of 2K + 1
// planes in registers fed from the ring, and the same arithmetic in the
// same order (lap3, leap2v, the reverse kernels' packed FMA for g), so the
// results are bitwise those of every other generation.
//
// The tensor maps cover the padded allocations (x from 0 to px, y and z
// with their H = K halo cells), so a tile's box starts at the field's
// (x0 - PX, y0 - K, z) = padded (x0, y0, z + K) (the first interior column
// X0 equals PX): in bounds, 16-byte aligned in x, and the cells outside
// the grid hold zero in memory (padding) or are filled with zero (beyond
// the allocation's extent), which is what the other generations read there.
// Planes past the end are clamped (their values are never used).
//
// Waits on the mbarriers are bounded; a wait that runs out raises error
// bit 8, the CTA stops at the next plane boundary, and thread 0 waits
// (with the full bound) for every copy still in flight before the CTA
// leaves.
#include <cuda.h>

#include "stencil_v3.cuh"

namespace ckfwi {
namespace {

__device__ __forceinline__ unsigned sa(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(bar)) : "memory");
}

__device__ __forceinline__ void bar_expect(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool bar_try(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(sa(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait with a short back-off; rounds < 0 gives up without looking
// (how a test makes a plane's wait run out); the drain before a CTA leaves
// always waits with the full bound, so no copy lands after it has gone
constexpr long long DRAIN_ROUNDS = 1LL << 22;
__device__ __forceinline__ bool bar_wait(uint64_t* bar, unsigned parity, long long rounds)
{
    if (rounds < 0) return false;
    for (int i = 0; i < 4; ++i)
        if (bar_try(bar, parity)) return true;
    for (long long i = 0; i < rounds; ++i) {
        __nanosleep(32);
        if (bar_try(bar, parity)) return true;
    }
    return false;
}

__device__ __forceinline__ void tile3(void* dst, const CUtensorMap* tm, int x, int y, int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(sa(dst)),
        "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(z), "r"(sa(bar))
        : "memory");
}

template <int K, int PF>
struct TQ {
    static constexpr int V = 4, TX = 8, TY = 16, D = PF;
    using G = G3<K, V, TX, TY>;
    static constexpr int RU = K + D + 1;                       // u tiles in the ring
    static constexpr int RP = D + 1;                           // point tiles of each point field
    static constexpr int UBYTES = G::TILE * 4;                 // one u box
    static constexpr int US = (UBYTES + 127) / 128 * 32;       // ring slot stride [floats], 128-byte multiple
    static constexpr int PT = G::BXP * TY;                     // floats of a point tile
    static constexpr int PBYTES = PT * 4;
    static constexpr size_t SMEM = (size_t)RU * US * 4 + 2 * (size_t)RP * PBYTES + RU * 8 + 128;
};

// first 128-byte aligned address of the dynamic shared memory
__device__ __forceinline__ unsigned char* align128(unsigned char* p)
{
    const unsigned a = sa(p);
    return p + ((128u - (a & 127u)) & 127u);
}

// CTAs an SM at order <= 8, set by the register cap: six with one plane of
// prefetch (31 KB of shared memory), five with two (39 KB)
template <int K, int PF> constexpr int tq_min_blocks() { return K <= 4 ? (PF == 1 ? 6 : 5) : 1; }

template <int K, int PF, int CK>
__global__ void __launch_bounds__(128, tq_min_blocks<K, PF>())
    fwdq_kernel(const FwdArgs a, const __grid_constant__ CUtensorMap tmu, const __grid_constant__ CUtensorMap tmp,
                const __grid_constant__ CUtensorMap tmw)
{
    using Q = TQ<K, PF>;
    using G = typename Q::G;
    constexpr int V = Q::V, TX = Q::TX, TY = Q::TY, D = Q::D, RU = Q::RU, RP = Q::RP;
    extern __shared__ unsigned char smq_raw[];
    __shared__ int abort_s[2];                  // a wait gave up at a step of this parity
    unsigned char* sm0 = align128(smq_raw);
    float* ring = reinterpret_cast<float*>(sm0);
    float* upr = ring + RU * Q::US;
    float* wr = upr + RP * Q::PT;
    uint64_t* bar = reinterpret_cast<uint64_t*>(wr + RP * Q::PT);

    const int bxi = blockIdx.x, byi = blockIdx.y, bzi = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int nz = a.g.nz, ny = a.g.ny, nx = a.g.nx;
    const int px = (int)a.g.px, pxy = (int)a.g.pxy;
    const int xb = bxi * G::BXP, yb = byi * TY;
    const int x0 = xb + V * tx;
    const int y = yb + ty;

    if (a.smp.n > 0) {   // receiver sampling of u^n by the first threads of the grid
        const int gt = ((bzi * gridDim.y + byi) * gridDim.x + bxi) * (TX * TY) + tid;
        if (gt < a.smp.n) {
            float acc = 0.0f;
            for (int i = 0; i < a.smp.nst; ++i)
                acc = __fmaf_rn(a.smp.wt[gt * a.smp.nst + i], __ldg(a.u + a.smp.idx[gt * a.smp.nst + i]), acc);
            a.smp.out[gt] = acc;
        }
    }

    const int z0 = bzi * a.zlen;
    if (z0 >= nz) return;                       // the whole CTA: no copy issued yet
    const int z1 = min(z0 + a.zlen, nz);
    const int nstep = z1 - z0;
    const bool rowact = y < ny;
    const bool cload = rowact && x0 < nx;
    const bool full = rowact && x0 + V <= nx;
    const int col = y * px + x0;
    const int cs = (ty + K) * G::RX + G::PX + V * tx;   // the thread's vector in a u tile
    const int ps = ty * G::BXP + V * tx;                // and in a point tile
    float ecol[V];
#pragma unroll
    for (int i = 0; i < V; ++i)
        ecol[i] = (rowact && x0 + i < nx) ? __fadd_rn(a.eta[nz + y], a.eta[nz + ny + x0 + i]) : 0.0f;
    Inj3<V> ij;
    ij.init(a.src, y, x0, nx, rowact);
    const int zqmax = nz + K - 1;
    const long long rounds = a.wait_limit;

    // Copy group g (g = 0, 1, ...): u plane z0 + g into slot g % RU and, for
    // g >= K, the point planes z0 + g - K into point slot (g - K) % RP, all
    // on barrier g % RU, whose phase (g / RU) it completes.
    auto issue = [&](int g) {
        uint64_t* b = bar + g % RU;
        const bool pts = g >= K;
        bar_expect(b, Q::UBYTES + (pts ? 2 * Q::PBYTES : 0));
        tile3(ring + (g % RU) * Q::US, &tmu, xb, yb, min(z0 + g, zqmax) + K, b);
        if (pts) {
            const int zp = min(z0 + g - K, z1 - 1) + K, s = (g - K) % RP;
            tile3(upr + s * Q::PT, &tmp, xb + G::PX, yb + K, zp, b);
            tile3(wr + s * Q::PT, &tmw, xb + G::PX, yb + K, zp, b);
        }
    };
    auto wait_group = [&](int g) { return bar_wait(bar + g % RU, (unsigned)((g / RU) & 1), rounds); };

    if (tid == 0) {
        abort_s[0] = abort_s[1] = 0;
        for (int s = 0; s < RU; ++s) bar_init(bar + s);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int g = 0; g < K + D; ++g) issue(g);
    }
    __syncthreads();
    int issued = K + D;                          // groups 0 .. issued - 1 are in flight or done

    // the queue: planes z0 - K .. z0 - 1 straight from global memory, planes
    // z0 .. z0 + K - 1 from the ring once their groups land
    float q[2 * K + 1][V];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        if (cload) gld<V>(q[i], a.u + (z0 - K + i) * pxy + col);
        else vzero<V>(q[i]);
    }
    int g0 = 0;
    while (g0 < K && wait_group(g0)) ++g0;
    if (g0 < K) abort_s[0] = 1;
    bool aborted = false;                        // the same in every thread: read after one barrier
    int confirmed = g0;                          // groups 0 .. confirmed - 1 are known complete
#pragma unroll
    for (int i = 0; i < K; ++i) sld<V>(q[K + i], ring + i * Q::US + cs);

    int step = 0;
    for (; step < nstep; ++step) {
        const int z = z0 + step;
        // the group of u plane z + K and point plane z
        // a wait that gave up flags this step's slot (step & 1): a thread one
        // step ahead writes the other slot, so all leave at the same step
        if (!wait_group(step + K)) abort_s[step & 1] = 1;
        __syncthreads();                        // every thread is past step - 1: its slots are free
        if (abort_s[step & 1]) {
            aborted = true;
            break;
        }
        confirmed = step + K + 1;
        if (tid == 0) issue(step + K + D);      // into the slots step - 1 read
        issued = step + K + D + 1;
        sld<V>(q[2 * K], ring + ((step + K) % RU) * Q::US + cs);
        const float* sm = ring + (step % RU) * Q::US;
        if (cload) {
            float upv[V], wv[V];
            sld<V>(upv, upr + (step % RP) * Q::PT + ps);
            sld<V>(wv, wr + (step % RP) * Q::PT + ps);
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
    }
    // no copy may land after the CTA has left: wait for the groups not yet
    // confirmed (bounded); a wait that ran out is reported
    if (tid == 0) {
        bool drained = true;
        for (int g = confirmed; g < issued; ++g)
            drained = bar_wait(bar + g % RU, (unsigned)((g / RU) & 1), DRAIN_ROUNDS) && drained;
        if (aborted || !drained) atomicOr(a.err, 8);
    }
}

template <int K, int PF, int CK>
cudaError_t fwdq_go(const FwdArgs& a, const CUtensorMap& tu, const CUtensorMap& tp, const CUtensorMap& tw,
                    cudaStream_t s)
{
    using Q = TQ<K, PF>;
    using G = typename Q::G;
    const dim3 blk(Q::TX, Q::TY, 1);
    const dim3 grd((a.g.nx + G::BXP - 1) / G::BXP, (a.g.ny + Q::TY - 1) / Q::TY, (a.g.nz + a.zlen - 1) / a.zlen);
    cudaError_t e = cudaFuncSetAttribute(fwdq_kernel<K, PF, CK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Q::SMEM);
    if (e != cudaSuccess) return e;
    fwdq_kernel<K, PF, CK><<<grd, blk, Q::SMEM, s>>>(a, tu, tp, tw);
    return cudaGetLastError();
}

template <int K, int PF>
cudaError_t fwdq_k(const FwdArgs& a, const CUtensorMap& tu, const CUtensorMap& tp, const CUtensorMap& tw, int ck,
                   cudaStream_t s)
{
    switch (ck) {
    case CK_NONE: return fwdq_go<K, PF, CK_NONE>(a, tu, tp, tw, s);
    case CK_FP32: return fwdq_go<K, PF, CK_FP32>(a, tu, tp, tw, s);
    case CK_BF16: return fwdq_go<K, PF, CK_BF16>(a, tu, tp, tw, s);
    case CK_FP16: return fwdq_go<K, PF, CK_FP16>(a, tu, tp, tw, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int K>
cudaError_t fwdq_p(const FwdArgs& a, const CUtensorMap& tu, const CUtensorMap& tp, const CUtensorMap& tw, int pf,
                   int ck, cudaStream_t s)
{
    return pf == 2 ? fwdq_k<K, 2>(a, tu, tp, tw, ck, s) : fwdq_k<K, 1>(a, tu, tp, tw, ck, s);
}

// The reverse step's gradient half: g += lam^{j-1} (lap u^{j-1} + Q^T s^{j-1}),
// with the same ring and queue of u^{j-1} as the forward step and point
// tiles of lam^{j-1} and g.  (The lam half, lam^{j-1} from lam^j and
// lam^{j+1}, is the forward step's arithmetic with the adjoint injection, so
// fwdq_kernel computes it.)  The arithmetic is the fused reverse kernels':
// the same Laplacian and injection order and one packed FMA, so g is
// bitwise theirs.
template <int K, int PF>
__global__ void __launch_bounds__(128, tq_min_blocks<K, PF>())
    gradq_kernel(const AdjArgs a, const __grid_constant__ CUtensorMap tmu, const __grid_constant__ CUtensorMap tml,
                 const __grid_constant__ CUtensorMap tmg)
{
    using Q = TQ<K, PF>;
    using G = typename Q::G;
    constexpr int V = Q::V, TX = Q::TX, TY = Q::TY, D = Q::D, RU = Q::RU, RP = Q::RP;
    extern __shared__ unsigned char smq_raw[];
    __shared__ int abort_s[2];                  // a wait gave up at a step of this parity
    unsigned char* sm0 = align128(smq_raw);
    float* ring = reinterpret_cast<float*>(sm0);
    float* lr = ring + RU * Q::US;
    float* gr = lr + RP * Q::PT;
    uint64_t* bar = reinterpret_cast<uint64_t*>(gr + RP * Q::PT);

    const int bxi = blockIdx.x, byi = blockIdx.y, bzi = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int nz = a.g.nz, ny = a.g.ny, nx = a.g.nx;
    const int px = (int)a.g.px, pxy = (int)a.g.pxy;
    const int xb = bxi * G::BXP, yb = byi * TY;
    const int x0 = xb + V * tx;
    const int y = yb + ty;
    const int z0 = bzi * a.zlen;
    if (z0 >= nz) return;
    const int z1 = min(z0 + a.zlen, nz);
    const int nstep = z1 - z0;
    const bool rowact = y < ny;
    const bool cload = rowact && x0 < nx;
    const bool full = rowact && x0 + V <= nx;
    const int col = y * px + x0;
    const int cs = (ty + K) * G::RX + G::PX + V * tx;
    const int ps = ty * G::BXP + V * tx;
    Inj3<V> is;
    is.init(a.src, y, x0, nx, rowact);
    const int zqmax = nz + K - 1;
    const long long rounds = a.wait_limit;
    const float* u = static_cast<const float*>(a.u);

    auto issue = [&](int g) {
        uint64_t* b = bar + g % RU;
        const bool pts = g >= K;
        bar_expect(b, Q::UBYTES + (pts ? 2 * Q::PBYTES : 0));
        tile3(ring + (g % RU) * Q::US, &tmu, xb, yb, min(z0 + g, zqmax) + K, b);
        if (pts) {
            const int zp = min(z0 + g - K, z1 - 1) + K, sl = (g - K) % RP;
            tile3(lr + sl * Q::PT, &tml, xb + G::PX, yb + K, zp, b);
            tile3(gr + sl * Q::PT, &tmg, xb + G::PX, yb + K, zp, b);
        }
    };
    auto wait_group = [&](int g) { return bar_wait(bar + g % RU, (unsigned)((g / RU) & 1), rounds); };

    if (tid == 0) {
        abort_s[0] = abort_s[1] = 0;
        for (int sl = 0; sl < RU; ++sl) bar_init(bar + sl);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int g = 0; g < K + D; ++g) issue(g);
    }
    __syncthreads();
    int issued = K + D;
    float q[2 * K + 1][V];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        if (cload) gld<V>(q[i], u + (z0 - K + i) * pxy + col);
        else vzero<V>(q[i]);
    }
    int g0 = 0;
    while (g0 < K && wait_group(g0)) ++g0;
    if (g0 < K) abort_s[0] = 1;
    bool aborted = false;                        // the same in every thread: read after one barrier
    int confirmed = g0;
#pragma unroll
    for (int i = 0; i < K; ++i) sld<V>(q[K + i], ring + i * Q::US + cs);

    for (int step = 0; step < nstep; ++step) {
        const int z = z0 + step;
        if (!wait_group(step + K)) abort_s[step & 1] = 1;
        __syncthreads();
        if (abort_s[step & 1]) {
            aborted = true;
            break;
        }
        confirmed = step + K + 1;
        if (tid == 0) issue(step + K + D);
        issued = step + K + D + 1;
        sld<V>(q[2 * K], ring + ((step + K) % RU) * Q::US + cs);
        const float* sm = ring + (step % RU) * Q::US;
        if (cload) {
            float lv[V], gv[V];
            sld<V>(lv, lr + (step % RP) * Q::PT + ps);
            sld<V>(gv, gr + (step % RP) * Q::PT + ps);
            float su[V];
            lap3<K, V, TX, TY>(su, q, sm, tx, ty, a.c);
            is.add(su, a.src, z);
            float gn[V];
#pragma unroll
            for (int p = 0; p < V / 2; ++p) {
                const int i = 2 * p;
                const float2 gg = __ffma2_rn(f2(lv[i], lv[i + 1]), f2(su[i], su[i + 1]), f2(gv[i], gv[i + 1]));
                gn[i] = gg.x;
                gn[i + 1] = gg.y;
            }
            const long long o = (long long)z * pxy + col;
            if (full) {
                vst<V>(a.gacc + o, gn);
            } else {
#pragma unroll
                for (int i = 0; i < V; ++i)
                    if (x0 + i < nx) a.gacc[o + i] = gn[i];
            }
        }
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) {
#pragma unroll
            for (int k = 0; k < V; ++k) q[i][k] = q[i + 1][k];
        }
    }
    if (tid == 0) {
        bool drained = true;
        for (int g = confirmed; g < issued; ++g)
            drained = bar_wait(bar + g % RU, (unsigned)((g / RU) & 1), DRAIN_ROUNDS) && drained;
        if (aborted || !drained) atomicOr(a.err, 8);
    }
}

template <int K, int PF>
cudaError_t gradq_go(const AdjArgs& a, const CUtensorMap& tu, const CUtensorMap& tl, const CUtensorMap& tg,
                     cudaStream_t s)
{
    using Q = TQ<K, PF>;
    using G = typename Q::G;
    const dim3 blk(Q::TX, Q::TY, 1);
    const dim3 grd((a.g.nx + G::BXP - 1) / G::BXP, (a.g.ny + Q::TY - 1) / Q::TY, (a.g.nz + a.zlen - 1) / a.zlen);
    cudaError_t e = cudaFuncSetAttribute(gradq_kernel<K, PF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Q::SMEM);
    if (e != cudaSuccess) return e;
    gradq_kernel<K, PF><<<grd, blk, Q::SMEM, s>>>(a, tu, tl, tg);
    return cudaGetLastError();
}

template <int K>
cudaError_t gradq_p(const AdjArgs& a, const CUtensorMap& tu, const CUtensorMap& tl, const CUtensorMap& tg, int pf,
                    cudaStream_t s)
{
    return pf == 2 ? gradq_go<K, 2>(a, tu, tl, tg, s) : gradq_go<K, 1>(a, tu, tl, tg, s);
}

}  // namespace

bool tq_supported(int dims, int K, const Tile& t)
{
    return dims == 3 && t.ver == 8 && (K == 1 || K == 2 || K == 4 || K == 8) && t.bx == 32 && t.by == 16 &&
           t.vec == 4 && t.zlen >= 1 && t.pf >= 0 && t.pf <= 2;
}

int tq_box_x(int K) { return 32 + 2 * (K <= 4 ? 4 : 8); }
int tq_box_y(int K) { return 16 + 2 * K; }

cudaError_t launch_fwdq(const FwdArgs& a, const CUtensorMap& tu, const CUtensorMap& tp, const CUtensorMap& tw,
                        const Tile& t, int K, int ck, cudaStream_t s)
{
    if (!v3_fits(a.g, K) || !tq_supported(a.g.dims, K, t)) return cudaErrorInvalidValue;
    // the boxes assume the first interior column at PX and H = K halo cells
    if (a.g.X0 != (K <= 4 ? 4 : 8) || a.g.H != K) return cudaErrorInvalidValue;
    FwdArgs b = a;
    b.zlen = t.zlen;
    switch (K) {
    case 1: return fwdq_p<1>(b, tu, tp, tw, t.pf, ck, s);
    case 2: return fwdq_p<2>(b, tu, tp, tw, t.pf, ck, s);
    case 4: return fwdq_p<4>(b, tu, tp, tw, t.pf, ck, s);
    case 8: return fwdq_p<8>(b, tu, tp, tw, t.pf, ck, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adjq(const AdjArgs& a, const CUtensorMap* maps, const Tile& t, int K, cudaStream_t s)
{
    if (!v3_fits(a.g, K) || !tq_supported(a.g.dims, K, t)) return cudaErrorInvalidValue;
    if (a.g.X0 != (K <= 4 ? 4 : 8) || a.g.H != K) return cudaErrorInvalidValue;
    // the lam half: a forward step of the adjoint field with the adjoint injection
    FwdArgs f{};
    f.g = a.g;
    f.u = a.l1;
    f.up = a.l2;
    f.w = a.w;
    f.out = a.l0;
    f.eta = a.eta;
    f.hdt = a.hdt;
    for (int j = 0; j <= MAXK; ++j) f.c[j] = a.c[j];
    f.src = a.adj;
    f.smp.n = 0;
    f.ck_u = nullptr;
    f.ck_up = nullptr;
    f.err = a.err;
    f.wait_limit = a.wait_limit;
    cudaError_t e = launch_fwdq(f, maps[0], maps[1], maps[2], t, K, CK_NONE, s);
    if (e != cudaSuccess) return e;
    AdjArgs b = a;
    b.zlen = t.zlen;
    switch (K) {
    case 1: return gradq_p<1>(b, maps[3], maps[4], maps[5], t.pf, s);
    case 2: return gradq_p<2>(b, maps[3], maps[4], maps[5], t.pf, s);
    case 4: return gradq_p<4>(b, maps[3], maps[4], maps[5], t.pf, s);
    case 8: return gradq_p<8>(b, maps[3], maps[4], maps[5], t.pf, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ckfwi
