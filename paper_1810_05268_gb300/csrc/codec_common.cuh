// Pieces shared by the codec's two modes (codec.cu: fixed accuracy,
// codec_rate.cu: fixed rate): block geometry, the sequency order, the
// lifting transform, negabinary and block positions.  Each translation unit
// gets its own copy (anonymous namespace, constant-memory tables).
#pragma once
#include <cstdint>

#include "internal.h"

namespace ckfwi {
namespace {

constexpr uint32_t MAGIC = 0x31435442u;
constexpr int HDR = 16;
constexpr int CHUNK = 32;

template <int DIMS> struct Cfg {
    static constexpr int V = DIMS == 3 ? 64 : 16;
    static constexpr int MAXBITS = 2 + 32 * V;
    static constexpr int MAXW = (MAXBITS + 31) / 32;       // words of the longest block stream
    static constexpr int AREA = (MAXW + 3) / 4 * 4;        // a block's staging area (16-byte multiple)
};

struct Geo {
    int dims, nz, ny, nx, nbz, nby, nbx;
    long long nblocks, nchunks, table_words;
};

__host__ __device__ inline Geo make_geo(int dims, int nz, int ny, int nx)
{
    Geo G;
    G.dims = dims; G.nz = nz; G.ny = ny; G.nx = nx;
    G.nbz = (nz + 3) / 4;
    G.nby = dims == 3 ? (ny + 3) / 4 : 1;
    G.nbx = (nx + 3) / 4;
    G.nblocks = (long long)G.nbz * G.nby * G.nbx;
    G.nchunks = (G.nblocks + CHUNK - 1) / CHUNK;
    G.table_words = HDR + G.nchunks + (G.nblocks + 1) / 2;
    return G;
}

// Scratch of one fixed-accuracy compression, in 32-bit words: a counter of
// finished compaction CTAs, the payload words of every group of 1024 chunks
// and of every group of 32 chunks (accumulated by the encoder, read and
// reset to zero by the compaction), each chunk's word count, and each
// chunk's staging slot of CW = 32 AREA words (first the blocks' own streams,
// AREA words apart, then the chunk's bits assembled contiguously).
struct ScratchLayout {
    long long g2, g1, counts, stage, words;
    int cw;
};
constexpr ScratchLayout scratch_layout_for(int dims, long long nchunks)
{
    ScratchLayout L{};
    const long long ng1 = (nchunks + 31) / 32, ng2 = (nchunks + 1023) / 1024;
    L.cw = CHUNK * (dims == 3 ? Cfg<3>::AREA : Cfg<2>::AREA);
    L.g2 = 32;
    L.g1 = L.g2 + ng2;
    L.counts = (L.g1 + ng1 + 31) / 32 * 32;
    L.stage = (L.counts + nchunks + 63) / 64 * 64;
    L.words = L.stage + nchunks * L.cw;
    return L;
}
__host__ __device__ inline ScratchLayout scratch_layout(const Geo& G) { return scratch_layout_for(G.dims, G.nchunks); }
// words of the scratch that must hold zero before a compression (the
// counter and both group sums); a compression leaves them zero again
__host__ __device__ inline long long scratch_zero_words(const Geo& G) { return scratch_layout(G).counts; }

// sequency order, built at compile time from its definition
struct Perm { int p[64]; };
constexpr Perm make_perm(int dims)
{
    Perm r{};
    int key[64] = {};
    const int V = dims == 3 ? 64 : 16;
    for (int i = 0; i < V; ++i) {
        const int kz = dims == 3 ? i / 16 : i / 4;
        const int ky = dims == 3 ? (i / 4) % 4 : 0;
        const int kx = i % 4;
        key[i] = ((kz + ky + kx) << 12) | (kz << 8) | (ky << 4) | kx;
        r.p[i] = i;
    }
    for (int a = 0; a < V; ++a) {
        int best = a;
        for (int b = a + 1; b < V; ++b)
            if (key[r.p[b]] < key[r.p[best]]) best = b;
        const int t = r.p[a];
        r.p[a] = r.p[best];
        r.p[best] = t;
    }
    return r;
}

// inverse of the sequency order: the rank of coefficient i (shared-memory
// rows are addressed by it at run time, so no register array is ever
// indexed with a run-time value)
constexpr Perm make_rank(int dims)
{
    const Perm P = make_perm(dims);
    Perm r{};
    for (int k = 0; k < 64; ++k) r.p[k] = 0;
    for (int k = 0; k < (dims == 3 ? 64 : 16); ++k) r.p[P.p[k]] = k;
    return r;
}
__constant__ Perm c_rank3 = make_rank(3);
__constant__ Perm c_rank2 = make_rank(2);
template <int DIMS> __device__ __forceinline__ int rank_of(int i) { return DIMS == 3 ? c_rank3.p[i] : c_rank2.p[i]; }

__device__ __forceinline__ int32_t half_of(int32_t a) { return a >> 1; }  // arithmetic shift

__device__ __forceinline__ void lift_fwd(int32_t& x0, int32_t& x1, int32_t& x2, int32_t& x3)
{
    const uint32_t u0 = x0, u1 = x1, u2 = x2, u3 = x3;
    const int32_t d3 = (int32_t)(u3 - (u2 + u2) + u1);
    const int32_t d1 = (int32_t)(u1 - (uint32_t)half_of((int32_t)(u0 + u2)));
    const int32_t D = (int32_t)(u2 - u0);
    const int32_t S = (int32_t)(u0 + (uint32_t)half_of(D));
    x0 = S; x1 = D; x2 = d1; x3 = d3;
}

__device__ __forceinline__ void lift_inv(int32_t& a0, int32_t& a1, int32_t& a2, int32_t& a3)
{
    const int32_t S = a0, D = a1, d1 = a2, d3 = a3;
    const int32_t x0 = (int32_t)((uint32_t)S - (uint32_t)half_of(D));
    const int32_t x2 = (int32_t)((uint32_t)D + (uint32_t)x0);
    const int32_t x1 = (int32_t)((uint32_t)d1 + (uint32_t)half_of((int32_t)((uint32_t)x0 + (uint32_t)x2)));
    const int32_t x3 = (int32_t)((uint32_t)d3 + (uint32_t)x2 + (uint32_t)x2 - (uint32_t)x1);
    a0 = x0; a1 = x1; a2 = x2; a3 = x3;
}

template <int DIMS>
__device__ __forceinline__ void xform_fwd(int32_t (&b)[Cfg<DIMS>::V])
{
    if constexpr (DIMS == 3) {
#pragma unroll
        for (int r = 0; r < 16; ++r) lift_fwd(b[4 * r], b[4 * r + 1], b[4 * r + 2], b[4 * r + 3]);
#pragma unroll
        for (int z = 0; z < 4; ++z)
#pragma unroll
            for (int x = 0; x < 4; ++x)
                lift_fwd(b[16 * z + x], b[16 * z + 4 + x], b[16 * z + 8 + x], b[16 * z + 12 + x]);
#pragma unroll
        for (int r = 0; r < 16; ++r) lift_fwd(b[r], b[16 + r], b[32 + r], b[48 + r]);
    } else {
#pragma unroll
        for (int z = 0; z < 4; ++z) lift_fwd(b[4 * z], b[4 * z + 1], b[4 * z + 2], b[4 * z + 3]);
#pragma unroll
        for (int x = 0; x < 4; ++x) lift_fwd(b[x], b[4 + x], b[8 + x], b[12 + x]);
    }
}

template <int DIMS>
__device__ __forceinline__ void xform_inv(int32_t (&b)[Cfg<DIMS>::V])
{
    if constexpr (DIMS == 3) {
#pragma unroll
        for (int r = 0; r < 16; ++r) lift_inv(b[r], b[16 + r], b[32 + r], b[48 + r]);
#pragma unroll
        for (int z = 0; z < 4; ++z)
#pragma unroll
            for (int x = 0; x < 4; ++x)
                lift_inv(b[16 * z + x], b[16 * z + 4 + x], b[16 * z + 8 + x], b[16 * z + 12 + x]);
#pragma unroll
        for (int r = 0; r < 16; ++r) lift_inv(b[4 * r], b[4 * r + 1], b[4 * r + 2], b[4 * r + 3]);
    } else {
#pragma unroll
        for (int x = 0; x < 4; ++x) lift_inv(b[x], b[4 + x], b[8 + x], b[12 + x]);
#pragma unroll
        for (int z = 0; z < 4; ++z) lift_inv(b[4 * z], b[4 * z + 1], b[4 * z + 2], b[4 * z + 3]);
    }
}

__device__ __forceinline__ uint32_t nega(int32_t c) { return ((uint32_t)c + 0xAAAAAAAAu) ^ 0xAAAAAAAAu; }
__device__ __forceinline__ int32_t unnega(uint32_t n) { return (int32_t)((n ^ 0xAAAAAAAAu) - 0xAAAAAAAAu); }

__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }

// block coordinates and clamped sample positions
struct BlockPos { int bz, by, bx; };
__device__ __forceinline__ BlockPos block_pos(const Geo& G, long long b)
{
    BlockPos p;
    if (G.nblocks <= 0xFFFFFFFFll) {
        // 32-bit division (a 64-bit one costs several times as many instructions)
        const unsigned ub = (unsigned)b, nbx = (unsigned)G.nbx, nby = (unsigned)G.nby;
        const unsigned t = ub / nbx, bz = t / nby;
        p.bx = (int)(ub - t * nbx);
        p.by = (int)(t - bz * nby);
        p.bz = (int)bz;
        return p;
    }
    p.bx = (int)(b % G.nbx);
    const long long t = b / G.nbx;
    p.by = (int)(t % G.nby);
    p.bz = (int)(t / G.nby);
    return p;
}

// In-place transpose of a 32 x 32 bit matrix: on return a[p] bit r is the
// input a[r] bit p (five stages of block swaps: j = 16, 8, 4, 2, 1).  The
// half-word and byte swaps of the first two stages are byte permutes (two
// per pair of words); the last three use masks.
__device__ __forceinline__ void transpose32(uint32_t (&a)[32])
{
#pragma unroll
    for (int k = 0; k < 16; ++k) {          // j = 16: swap a[k] bits 16..31 with a[k+16] bits 0..15
        const uint32_t x = a[k], y = a[k + 16];
        a[k] = __byte_perm(x, y, 0x5410);
        a[k + 16] = __byte_perm(x, y, 0x7632);
    }
#pragma unroll
    for (int k = 0; k < 32; ++k) {          // j = 8: swap the odd bytes of a[k] with the even bytes of a[k+8]
        if (k & 8) continue;
        const uint32_t x = a[k], y = a[k + 8];
        a[k] = __byte_perm(x, y, 0x6240);
        a[k + 8] = __byte_perm(x, y, 0x7351);
    }
    constexpr uint32_t M[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int st = 2; st < 5; ++st) {
        const int j = 16 >> st;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            if (k & j) continue;
            const uint32_t t = ((a[k] >> j) ^ a[k + j]) & M[st];
            a[k] ^= t << j;
            a[k + j] ^= t;
        }
    }
}

template <int DIMS>
__device__ __forceinline__ void gather(const float* __restrict__ x, const CodecView& v, const BlockPos& bp,
                                       float (&f)[Cfg<DIMS>::V])
{
    const int xs = 4 * bp.bx;
    const bool vec = v.aligned && xs + 3 < v.nx;
    constexpr int ROWS = DIMS == 3 ? 16 : 4;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const int lz = DIMS == 3 ? r / 4 : r;
        const int ly = DIMS == 3 ? r % 4 : 0;
        const int z = min(4 * bp.bz + lz, v.nz - 1);
        const int y = DIMS == 3 ? min(4 * bp.by + ly, v.ny - 1) : 0;
        const float* row = x + (long long)z * v.pz + (long long)y * v.py;
        if (vec) {
            const float4 q = __ldg(reinterpret_cast<const float4*>(row + xs));
            f[4 * r] = q.x; f[4 * r + 1] = q.y; f[4 * r + 2] = q.z; f[4 * r + 3] = q.w;
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) f[4 * r + c] = __ldg(row + min(xs + c, v.nx - 1));
        }
    }
}

}  // namespace
}  // namespace ckfwi
