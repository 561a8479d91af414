// Batched forward and reverse steps: one launch advances every lane (shot)
// of a batch by one step.  Lane l owns CTAs start[l] .. start[l+1]-1 of a
// 1D grid, laid out like the grid of its own single-lane launch (x
// fastest, then y, then z runs); its arguments (geometry, fields,
// injection, sampling) are tab[l].  Each CTA finds its lane by binary
// search and stages the lane's arguments in shared memory.  The device
// code is the single-lane kernels' (stencil_body.cuh), so a lane's fields
// are bitwise those of a single-shot run.
#include "stencil_body.cuh"

namespace ckfwi {

template <int K, int DIMS, int BX, int BY, int CK>
__global__ void __launch_bounds__(BX * BY)
    fwd_batch_kernel(const FwdArgs* __restrict__ tab, const int* __restrict__ start, int nl)
{
    extern __shared__ float sm[];
    __shared__ __align__(16) FwdArgs a;
    const int b = stage_args(a, tab, start, nl);
    const int gx = (a.g.nx + BX - 1) / BX;
    const int gy = DIMS == 3 ? (a.g.ny + BY - 1) / BY : 1;
    fwd_body<K, DIMS, BX, BY, CK>(a, sm, b % gx, (b / gx) % gy, b / (gx * gy), gx, gy);
}

template <int K, int DIMS, int BX, int BY, class UT>
__global__ void __launch_bounds__(BX * BY)
    adj_batch_kernel(const AdjArgs* __restrict__ tab, const int* __restrict__ start, int nl)
{
    extern __shared__ float sm[];
    __shared__ __align__(16) AdjArgs a;
    const int b = stage_args(a, tab, start, nl);
    const int gx = (a.g.nx + BX - 1) / BX;
    const int gy = DIMS == 3 ? (a.g.ny + BY - 1) / BY : 1;
    adj_body<K, DIMS, BX, BY, UT>(a, sm, b % gx, (b / gx) % gy, b / (gx * gy));
}

namespace {

template <int K, int DIMS, int BX, int BY>
cudaError_t fwd_batch_go(const BatchLaunch<FwdArgs>& b, int ck, cudaStream_t s)
{
    const dim3 blk(BX, BY, 1), grd((unsigned)b.blocks, 1, 1);
    const size_t sh = smem_bytes<DIMS, BX, BY>(K, 1);
    switch (ck) {
    case CK_NONE: fwd_batch_kernel<K, DIMS, BX, BY, CK_NONE><<<grd, blk, sh, s>>>(b.tab, b.start, b.lanes); break;
    case CK_FP32: fwd_batch_kernel<K, DIMS, BX, BY, CK_FP32><<<grd, blk, sh, s>>>(b.tab, b.start, b.lanes); break;
    case CK_BF16: fwd_batch_kernel<K, DIMS, BX, BY, CK_BF16><<<grd, blk, sh, s>>>(b.tab, b.start, b.lanes); break;
    case CK_FP16: fwd_batch_kernel<K, DIMS, BX, BY, CK_FP16><<<grd, blk, sh, s>>>(b.tab, b.start, b.lanes); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int K, int DIMS, int BX, int BY>
cudaError_t adj_batch_go(const BatchLaunch<AdjArgs>& b, int ut, cudaStream_t s)
{
    const dim3 blk(BX, BY, 1), grd((unsigned)b.blocks, 1, 1);
    const size_t sh = smem_bytes<DIMS, BX, BY>(K, 2);
    switch (ut) {
    case U_FP32: adj_batch_kernel<K, DIMS, BX, BY, float><<<grd, blk, sh, s>>>(b.tab, b.start, b.lanes); break;
    case U_BF16: adj_batch_kernel<K, DIMS, BX, BY, __nv_bfloat16><<<grd, blk, sh, s>>>(b.tab, b.start, b.lanes); break;
    case U_FP16: adj_batch_kernel<K, DIMS, BX, BY, __half><<<grd, blk, sh, s>>>(b.tab, b.start, b.lanes); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int K>
cudaError_t fwd_batch_k(const BatchLaunch<FwdArgs>& b, const Tile& t, int ck, cudaStream_t s)
{
    if (b.dims == 3 && t.by < K) return cudaErrorInvalidValue;   // halo rows need BY >= K
    if (b.dims == 3) {
        if (t.bx == 32 && t.by == 4) return fwd_batch_go<K, 3, 32, 4>(b, ck, s);
        if (t.bx == 32 && t.by == 8) return fwd_batch_go<K, 3, 32, 8>(b, ck, s);
        if (t.bx == 32 && t.by == 16) return fwd_batch_go<K, 3, 32, 16>(b, ck, s);
    } else {
        if (t.bx == 128) return fwd_batch_go<K, 2, 128, 1>(b, ck, s);
        if (t.bx == 256) return fwd_batch_go<K, 2, 256, 1>(b, ck, s);
    }
    return cudaErrorInvalidValue;
}

template <int K>
cudaError_t adj_batch_k(const BatchLaunch<AdjArgs>& b, const Tile& t, int ut, cudaStream_t s)
{
    if (b.dims == 3 && t.by < K) return cudaErrorInvalidValue;   // halo rows need BY >= K
    if (b.dims == 3) {
        if (t.bx == 32 && t.by == 4) return adj_batch_go<K, 3, 32, 4>(b, ut, s);
        if (t.bx == 32 && t.by == 8) return adj_batch_go<K, 3, 32, 8>(b, ut, s);
        if (t.bx == 32 && t.by == 16) return adj_batch_go<K, 3, 32, 16>(b, ut, s);
    } else {
        if (t.bx == 128) return adj_batch_go<K, 2, 128, 1>(b, ut, s);
        if (t.bx == 256) return adj_batch_go<K, 2, 256, 1>(b, ut, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_fwd_batch(const BatchLaunch<FwdArgs>& b, const Tile& t, int K, int ck, cudaStream_t s)
{
    if (b.lanes < 1 || b.blocks < 1 || b.blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    switch (K) {
    case 1: return fwd_batch_k<1>(b, t, ck, s);
    case 2: return fwd_batch_k<2>(b, t, ck, s);
    case 4: return fwd_batch_k<4>(b, t, ck, s);
    case 8: return fwd_batch_k<8>(b, t, ck, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adj_batch(const BatchLaunch<AdjArgs>& b, const Tile& t, int K, int ut, cudaStream_t s)
{
    if (b.lanes < 1 || b.blocks < 1 || b.blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    switch (K) {
    case 1: return adj_batch_k<1>(b, t, ut, s);
    case 2: return adj_batch_k<2>(b, t, ut, s);
    case 4: return adj_batch_k<4>(b, t, ut, s);
    case 8: return adj_batch_k<8>(b, t, ut, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ckfwi
