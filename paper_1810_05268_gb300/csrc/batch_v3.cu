// Batched vector-blocked steps: one launch advances every lane (shot) of a
// batch by one step, each lane's CTAs laid out like its own single-lane
// grid (x fastest, then y, then z runs) and its arguments staged from a
// device table.  The device code is the single-shot kernels'
// (stencil_v3.cuh), so every lane's values are bitwise a single-shot run's.
#include "stencil_v3.cuh"

namespace ckfwi {
namespace {

template <int K, int V, int TX, int TY, int CK>
__global__ void __launch_bounds__(TX * TY)
    fwd3_batch_kernel(const FwdArgs* __restrict__ tab, const int* __restrict__ start, int nl)
{
    using G = G3<K, V, TX, TY>;
    extern __shared__ __align__(16) float smem3[];
    __shared__ __align__(16) FwdArgs a;
    const int b = stage_args(a, tab, start, nl);
    const int gx = (a.g.nx + G::BXP - 1) / G::BXP;
    const int gy = (a.g.ny + TY - 1) / TY;
    fwd3_body<K, V, TX, TY, CK>(a, smem3, b % gx, (b / gx) % gy, b / (gx * gy), gx, gy);
}

template <int K, int V, int TX, int TY, class UT>
__global__ void __launch_bounds__(TX * TY)
    adj3_batch_kernel(const AdjArgs* __restrict__ tab, const int* __restrict__ start, int nl)
{
    using G = G3<K, V, TX, TY>;
    extern __shared__ __align__(16) float smem3[];
    __shared__ __align__(16) AdjArgs a;
    const int b = stage_args(a, tab, start, nl);
    const int gx = (a.g.nx + G::BXP - 1) / G::BXP;
    const int gy = (a.g.ny + TY - 1) / TY;
    adj3_body<K, V, TX, TY, UT>(a, smem3, b % gx, (b / gx) % gy, b / (gx * gy));
}

template <int K, int V, int TX, int TY>
cudaError_t fwd3b_go(const BatchLaunch<FwdArgs>& b, int ck, cudaStream_t s)
{
    using G = G3<K, V, TX, TY>;
    const dim3 blk(TX, TY, 1), grd((unsigned)b.blocks, 1, 1);
    const size_t sh = 2 * (size_t)G::TILE * sizeof(float);
    switch (ck) {
    case CK_NONE: fwd3_batch_kernel<K, V, TX, TY, CK_NONE><<<grd, blk, sh, s>>>(b.tab, b.start, b.lanes); break;
    case CK_FP32: fwd3_batch_kernel<K, V, TX, TY, CK_FP32><<<grd, blk, sh, s>>>(b.tab, b.start, b.lanes); break;
    case CK_BF16: fwd3_batch_kernel<K, V, TX, TY, CK_BF16><<<grd, blk, sh, s>>>(b.tab, b.start, b.lanes); break;
    case CK_FP16: fwd3_batch_kernel<K, V, TX, TY, CK_FP16><<<grd, blk, sh, s>>>(b.tab, b.start, b.lanes); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int K, int V, int TX, int TY>
cudaError_t adj3b_go(const BatchLaunch<AdjArgs>& b, int ut, cudaStream_t s)
{
    using G = G3<K, V, TX, TY>;
    const dim3 blk(TX, TY, 1), grd((unsigned)b.blocks, 1, 1);
    const size_t sh = 4 * (size_t)G::TILE * sizeof(float);
    switch (ut) {
    case U_FP32: adj3_batch_kernel<K, V, TX, TY, float><<<grd, blk, sh, s>>>(b.tab, b.start, b.lanes); break;
    case U_BF16: adj3_batch_kernel<K, V, TX, TY, __nv_bfloat16><<<grd, blk, sh, s>>>(b.tab, b.start, b.lanes); break;
    case U_FP16: adj3_batch_kernel<K, V, TX, TY, __half><<<grd, blk, sh, s>>>(b.tab, b.start, b.lanes); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int K>
cudaError_t fwd3b_k(const BatchLaunch<FwdArgs>& b, const Tile& t, int ck, cudaStream_t s)
{
    if (t.vec == 4 && t.bx == 32 && t.by == 16) return fwd3b_go<K, 4, 8, 16>(b, ck, s);
    if (t.vec == 2 && t.bx == 32 && t.by == 16) return fwd3b_go<K, 2, 16, 16>(b, ck, s);
    return cudaErrorInvalidValue;
}

template <int K>
cudaError_t adj3b_k(const BatchLaunch<AdjArgs>& b, const Tile& t, int ut, cudaStream_t s)
{
    if (t.vec == 4 && t.bx == 32 && t.by == 16) return adj3b_go<K, 4, 8, 16>(b, ut, s);
    if (t.vec == 2 && t.bx == 32 && t.by == 16) return adj3b_go<K, 2, 16, 16>(b, ut, s);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_fwd3_batch(const BatchLaunch<FwdArgs>& b, const Tile& t, int K, int ck, cudaStream_t s)
{
    if (b.dims != 3 || b.lanes < 1 || b.blocks < 1 || b.blocks > 0x7fffffffLL || !v3_supported(3, K, t))
        return cudaErrorInvalidValue;
    switch (K) {
    case 1: return fwd3b_k<1>(b, t, ck, s);
    case 2: return fwd3b_k<2>(b, t, ck, s);
    case 4: return fwd3b_k<4>(b, t, ck, s);
    case 8: return fwd3b_k<8>(b, t, ck, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adj3_batch(const BatchLaunch<AdjArgs>& b, const Tile& t, int K, int ut, cudaStream_t s)
{
    if (b.dims != 3 || b.lanes < 1 || b.blocks < 1 || b.blocks > 0x7fffffffLL || !v3_supported(3, K, t))
        return cudaErrorInvalidValue;
    switch (K) {
    case 1: return adj3b_k<1>(b, t, ut, s);
    case 2: return adj3b_k<2>(b, t, ut, s);
    case 4: return adj3b_k<4>(b, t, ut, s);
    case 8: return adj3b_k<8>(b, t, ut, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ckfwi
