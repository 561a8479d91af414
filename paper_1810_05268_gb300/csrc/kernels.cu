// Forward and fused reverse time steps of the OT2 acoustic kernel
// (Sec. 6, Eq. "eqn:wave"): one launch per step of one shot.  The device
// code (register-queue z-march, shared-memory halos, difference-form
// Laplacian, fused imaging condition) is in stencil_body.cuh.
#include "stencil_body.cuh"

namespace ckfwi {

template <int K, int DIMS, int BX, int BY, int CK>
__global__ void __launch_bounds__(BX * BY) fwd_kernel(const FwdArgs a)
{
    extern __shared__ float sm[];
    fwd_body<K, DIMS, BX, BY, CK>(a, sm, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y);
}

template <int K, int DIMS, int BX, int BY, class UT>
__global__ void __launch_bounds__(BX * BY) adj_kernel(const AdjArgs a)
{
    extern __shared__ float sm[];
    adj_body<K, DIMS, BX, BY, UT>(a, sm, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ---------------------------------------------------------------- dispatch
namespace {
constexpr int N3 = 3;
constexpr int TILES3[N3][2] = {{32, 4}, {32, 8}, {32, 16}};
constexpr int N2 = 2;
constexpr int TILES2[N2] = {128, 256};

template <int K, int DIMS, int BX, int BY>
cudaError_t fwd_go(const FwdArgs& a, int ck, cudaStream_t s)
{
    dim3 blk(BX, BY, 1);
    dim3 grd((a.g.nx + BX - 1) / BX, DIMS == 3 ? (a.g.ny + BY - 1) / BY : 1,
             (a.g.nz + a.zlen - 1) / a.zlen);
    const size_t sh = smem_bytes<DIMS, BX, BY>(K, 1);
    switch (ck) {
    case CK_NONE: fwd_kernel<K, DIMS, BX, BY, CK_NONE><<<grd, blk, sh, s>>>(a); break;
    case CK_FP32: fwd_kernel<K, DIMS, BX, BY, CK_FP32><<<grd, blk, sh, s>>>(a); break;
    case CK_BF16: fwd_kernel<K, DIMS, BX, BY, CK_BF16><<<grd, blk, sh, s>>>(a); break;
    case CK_FP16: fwd_kernel<K, DIMS, BX, BY, CK_FP16><<<grd, blk, sh, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int K, int DIMS, int BX, int BY>
cudaError_t adj_go(const AdjArgs& a, int ut, cudaStream_t s)
{
    dim3 blk(BX, BY, 1);
    dim3 grd((a.g.nx + BX - 1) / BX, DIMS == 3 ? (a.g.ny + BY - 1) / BY : 1,
             (a.g.nz + a.zlen - 1) / a.zlen);
    const size_t sh = smem_bytes<DIMS, BX, BY>(K, 2);
    switch (ut) {
    case U_FP32: adj_kernel<K, DIMS, BX, BY, float><<<grd, blk, sh, s>>>(a); break;
    case U_BF16: adj_kernel<K, DIMS, BX, BY, __nv_bfloat16><<<grd, blk, sh, s>>>(a); break;
    case U_FP16: adj_kernel<K, DIMS, BX, BY, __half><<<grd, blk, sh, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int K>
cudaError_t fwd_k(const FwdArgs& a, const Tile& t, int ck, cudaStream_t s)
{
    if (a.g.dims == 3 && t.by < K) return cudaErrorInvalidValue;   // halo rows need BY >= K
    if (a.g.dims == 3) {
        if (t.bx == 32 && t.by == 4) return fwd_go<K, 3, 32, 4>(a, ck, s);
        if (t.bx == 32 && t.by == 8) return fwd_go<K, 3, 32, 8>(a, ck, s);
        if (t.bx == 32 && t.by == 16) return fwd_go<K, 3, 32, 16>(a, ck, s);
    } else {
        if (t.bx == 128) return fwd_go<K, 2, 128, 1>(a, ck, s);
        if (t.bx == 256) return fwd_go<K, 2, 256, 1>(a, ck, s);
    }
    return cudaErrorInvalidValue;
}

template <int K>
cudaError_t adj_k(const AdjArgs& a, const Tile& t, int ut, cudaStream_t s)
{
    if (a.g.dims == 3 && t.by < K) return cudaErrorInvalidValue;   // halo rows need BY >= K
    if (a.g.dims == 3) {
        if (t.bx == 32 && t.by == 4) return adj_go<K, 3, 32, 4>(a, ut, s);
        if (t.bx == 32 && t.by == 8) return adj_go<K, 3, 32, 8>(a, ut, s);
        if (t.bx == 32 && t.by == 16) return adj_go<K, 3, 32, 16>(a, ut, s);
    } else {
        if (t.bx == 128) return adj_go<K, 2, 128, 1>(a, ut, s);
        if (t.bx == 256) return adj_go<K, 2, 256, 1>(a, ut, s);
    }
    return cudaErrorInvalidValue;
}
}  // namespace

int tile_count(int dims) { return dims == 3 ? N3 : N2; }

Tile tile_at(int dims, int i, int zlen)
{
    Tile t;
    if (dims == 3) {
        t.bx = TILES3[i][0];
        t.by = TILES3[i][1];
    } else {
        t.bx = TILES2[i];
        t.by = 1;
    }
    t.zlen = zlen;
    return t;
}

bool tile_supported(int dims, int K, const Tile& t)
{
    // the x and y halos are staged by the first K threads of a row / column
    if (t.bx < K || (dims == 3 && t.by < K)) return false;
    for (int i = 0; i < tile_count(dims); ++i) {
        Tile u = tile_at(dims, i, t.zlen);
        if (u.bx == t.bx && u.by == t.by) return t.zlen >= 1;
    }
    return false;
}

cudaError_t launch_fwd(const FwdArgs& a, const Tile& t, int K, int ck, cudaStream_t s)
{
    FwdArgs b = a;
    b.zlen = t.zlen;
    switch (K) {
    case 1: return fwd_k<1>(b, t, ck, s);
    case 2: return fwd_k<2>(b, t, ck, s);
    case 4: return fwd_k<4>(b, t, ck, s);
    case 8: return fwd_k<8>(b, t, ck, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adj(const AdjArgs& a, const Tile& t, int K, int ut, cudaStream_t s)
{
    AdjArgs b = a;
    b.zlen = t.zlen;
    switch (K) {
    case 1: return adj_k<1>(b, t, ut, s);
    case 2: return adj_k<2>(b, t, ut, s);
    case 4: return adj_k<4>(b, t, ut, s);
    case 8: return adj_k<8>(b, t, ut, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ckfwi
