// Vector-blocked forward and fused reverse steps for 3D grids, one shot per
// launch.  The device code and its design notes are in stencil_v3.cuh.
#include "stencil_v3.cuh"

namespace ckfwi {
namespace {

template <int K, int V, int TX, int TY, int CK>
__global__ void __launch_bounds__(TX * TY) fwd3_kernel(const FwdArgs a)
{
    extern __shared__ __align__(16) float smem3[];
    fwd3_body<K, V, TX, TY, CK>(a, smem3, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y);
}

// Four-point FP32 reverse steps up to order 8 are capped at 168 registers,
// so that three 128-thread CTAs fit an SM (8 bytes of spill at order 8; 236
// registers and two CTAs uncapped): the step is latency-bound at 8 warps.
// The 16-bit variants spill inside the plane loop under the cap and stay
// uncapped.
template <int K, int V, class UT>
constexpr int adj3_min_blocks() { return V == 4 && K <= 4 && std::is_same<UT, float>::value ? 3 : 1; }

template <int K, int V, int TX, int TY, class UT>
__global__ void __launch_bounds__(TX * TY, adj3_min_blocks<K, V, UT>()) adj3_kernel(const AdjArgs a)
{
    extern __shared__ __align__(16) float smem3[];
    adj3_body<K, V, TX, TY, UT>(a, smem3, blockIdx.x, blockIdx.y, blockIdx.z);
}


// ------------------------------------------------------------- dispatch
// (V, TX, TY) shapes; Tile.bx = V * TX, Tile.by = TY, Tile.vec = V
struct Shape3 {
    int v, tx, ty;
};
constexpr Shape3 SHAPES3[] = {{4, 8, 16}, {2, 16, 16}};
constexpr int NSHAPES3 = sizeof(SHAPES3) / sizeof(SHAPES3[0]);

template <int K, int V, int TX, int TY>
cudaError_t fwd3_go(const FwdArgs& a, int ck, cudaStream_t s)
{
    using G = G3<K, V, TX, TY>;
    const dim3 blk(TX, TY, 1);
    const dim3 grd((a.g.nx + G::BXP - 1) / G::BXP, (a.g.ny + TY - 1) / TY, (a.g.nz + a.zlen - 1) / a.zlen);
    const size_t sh = 2 * (size_t)G::TILE * sizeof(float);
    switch (ck) {
    case CK_NONE: fwd3_kernel<K, V, TX, TY, CK_NONE><<<grd, blk, sh, s>>>(a); break;
    case CK_FP32: fwd3_kernel<K, V, TX, TY, CK_FP32><<<grd, blk, sh, s>>>(a); break;
    case CK_BF16: fwd3_kernel<K, V, TX, TY, CK_BF16><<<grd, blk, sh, s>>>(a); break;
    case CK_FP16: fwd3_kernel<K, V, TX, TY, CK_FP16><<<grd, blk, sh, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int K, int V, int TX, int TY>
cudaError_t adj3_go(const AdjArgs& a, int ut, cudaStream_t s)
{
    using G = G3<K, V, TX, TY>;
    const dim3 blk(TX, TY, 1);
    const dim3 grd((a.g.nx + G::BXP - 1) / G::BXP, (a.g.ny + TY - 1) / TY, (a.g.nz + a.zlen - 1) / a.zlen);
    const size_t sh = 4 * (size_t)G::TILE * sizeof(float);
    switch (ut) {
    case U_FP32: adj3_kernel<K, V, TX, TY, float><<<grd, blk, sh, s>>>(a); break;
    case U_BF16: adj3_kernel<K, V, TX, TY, __nv_bfloat16><<<grd, blk, sh, s>>>(a); break;
    case U_FP16: adj3_kernel<K, V, TX, TY, __half><<<grd, blk, sh, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int K>
cudaError_t fwd3_k(const FwdArgs& a, const Tile& t, int ck, cudaStream_t s)
{
    if (t.vec == 4 && t.bx == 32 && t.by == 16) return fwd3_go<K, 4, 8, 16>(a, ck, s);
    if (t.vec == 2 && t.bx == 32 && t.by == 16) return fwd3_go<K, 2, 16, 16>(a, ck, s);
    return cudaErrorInvalidValue;
}

template <int K>
cudaError_t adj3_k(const AdjArgs& a, const Tile& t, int ut, cudaStream_t s)
{
    if (t.vec == 4 && t.bx == 32 && t.by == 16) return adj3_go<K, 4, 8, 16>(a, ut, s);
    if (t.vec == 2 && t.bx == 32 && t.by == 16) return adj3_go<K, 2, 16, 16>(a, ut, s);
    return cudaErrorInvalidValue;
}

}  // namespace

int v3_shape_count() { return NSHAPES3; }

Tile v3_tile_at(int i, int zlen)
{
    Tile t;
    t.bx = SHAPES3[i].v * SHAPES3[i].tx;
    t.by = SHAPES3[i].ty;
    t.zlen = zlen;
    t.ver = 3;
    t.vec = SHAPES3[i].v;
    return t;
}

bool v3_fits(const FieldGeom& g, int K)
{
    // element offsets inside a field are 32-bit
    return g.dims == 3 && (long long)(g.nz + 2 * K + 1) * g.pxy < 0x7fffffffLL;
}

bool v3_supported(int dims, int K, const Tile& t)
{
    if (dims != 3 || t.ver != 3 || t.zlen < 1 || t.by < K) return false;
    if (K != 1 && K != 2 && K != 4 && K != 8) return false;
    for (int i = 0; i < NSHAPES3; ++i) {
        const Tile u = v3_tile_at(i, t.zlen);
        if (u.bx == t.bx && u.by == t.by && u.vec == t.vec) return true;
    }
    return false;
}

cudaError_t launch_fwd3(const FwdArgs& a, const Tile& t, int K, int ck, cudaStream_t s)
{
    FwdArgs b = a;
    b.zlen = t.zlen;
    if (!v3_fits(a.g, K) || !v3_supported(a.g.dims, K, t)) return cudaErrorInvalidValue;
    switch (K) {
    case 1: return fwd3_k<1>(b, t, ck, s);
    case 2: return fwd3_k<2>(b, t, ck, s);
    case 4: return fwd3_k<4>(b, t, ck, s);
    case 8: return fwd3_k<8>(b, t, ck, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adj3(const AdjArgs& a, const Tile& t, int K, int ut, cudaStream_t s)
{
    AdjArgs b = a;
    b.zlen = t.zlen;
    if (!v3_fits(a.g, K) || !v3_supported(a.g.dims, K, t)) return cudaErrorInvalidValue;
    switch (K) {
    case 1: return adj3_k<1>(b, t, ut, s);
    case 2: return adj3_k<2>(b, t, ut, s);
    case 4: return adj3_k<4>(b, t, ut, s);
    case 8: return adj3_k<8>(b, t, ut, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ckfwi

