// Fixed-accuracy block-transform codec for checkpoints held in HBM.
//
// The paper compresses checkpoints with ZFP in fixed-tolerance mode, an
// absolute point-wise error bound (Sec. 2.2 "Lossy Compression"); Sec. 4
// turns the ratio F into F times more checkpoint slots.  This codec is of
// the same family and is specified here in full (it is not ZFP and not
// bit-compatible with it):
//
//  blocks   4^d cubes (2D: 4x4 over z, x), block b = (bz*nby + by)*nbx + bx;
//           a partial block repeats the last valid sample along each axis.
//  zero     max |x| <= tol_f (largest float <= tol): a single 0 bit.
//  integers Emax = max exponent max(biased,1)-127 over non-zero values;
//           i = trunc(x 2^(23-Emax)) from the bits, |i| < 2^24.
//  lifting  per 4-vector along x, then y, then z, 32-bit wrap-around:
//           d3 = x3 - 2x2 + x1, d1 = x1 - ((x0+x2)>>1), D = x2 - x0,
//           S = x0 + (D>>1)  ->  (S, D, d1, d3); exactly invertible.
//  order    by (kz+ky+kx, kz, ky, kx); negabinary n = (c + A) ^ A,
//           A = 0xAAAAAAAA.
//  planes   ptop = highest set bit of all n; T = floor(tol_f 2^(23-Emax));
//           pbot = first plane, from min(ptop, max(0, floor(log2 T) - 1))
//           down to 0, whose truncation reproduces every i within T - 2
//           (closed loop, so |x - x_hat| <= tol on every value); T < 2 or
//           Emax >= 126: raw block.
//  stream   1 0 Emax+127(8) ptop(5) pbot(5), then planes ptop..pbot: the
//           bits of the s significant coefficients verbatim, then group
//           tests (1 = some coefficient >= s is set: its bits follow up to
//           and including the first set one; 0 = none).  Raw: 1 1, then the
//           float bit patterns.  A coded stream longer than the raw form
//           (2 + 32 V bits) is replaced by it.  LSB-first in 32-bit words.
//  container [16 header words][chunk word offsets][uint16 block bit sizes]
//           [payload]; a chunk is 32 consecutive blocks and starts on a
//           word boundary.
//
// GPU layout of the work: one thread encodes / decodes one block; a warp
// owns one chunk, so block bit offsets inside a chunk come from a warp scan
// of the size table.  Compression runs in two launches:
//  1. encode: every thread codes its block through its own shared-memory
//     column into its own area of the chunk's staging slot in scratch; the
//     warp assembles its chunk's bits contiguously in shared memory and
//     writes them back over the slot, with the chunk's word count, which it
//     also adds to the sums of its group of 32 and of 1024 chunks;
//  2. compact: a small CTA per 4 chunks copies them from staging to the
//     payload at offsets formed from at most (chunks / 1024) + 62 group sums
//     and chunk counts (linear total work); CTA 0 writes the header, the
//     last CTA resets the group sums.
// The pool position of a stream is read from and written to device memory,
// so a schedule of compressions and decompressions runs without host
// synchronisation; running out of pool raises an error bit and the stream
// is not written.  The scratch's counter and group sums must be zero before
// the first compression; every compression leaves them zero.
#include <cstdint>
#include <utility>

#include "codec_common.cuh"

namespace ckfwi {
namespace {

constexpr uint32_t VERSION = 1u;
constexpr int GUARD = 1;
constexpr int ENC_THREADS = 64;
constexpr int DEC_THREADS = 128;



// Bit writer into a block's stream area in global memory (MAXW contiguous
// words, in the chunk's staging slot); words past MAXW are counted but not
// stored (such a stream is replaced by the raw form).
template <int DIMS>
struct BitW {
    static constexpr int MW = Cfg<DIMS>::MAXW;
    uint32_t* w;
    unsigned long long acc;
    int nacc;
    int nw;
    __device__ __forceinline__ void store(uint32_t v)
    {
        if (nw < MW) w[nw] = v;
        ++nw;
    }
    __device__ __forceinline__ void put(uint32_t v, int n)   // n <= 32, v < 2^n
    {
        acc |= (unsigned long long)v << nacc;
        nacc += n;
        if (nacc >= 32) {
            store((uint32_t)acc);
            acc >>= 32;
            nacc -= 32;
        }
    }
    __device__ __forceinline__ void put64(unsigned long long v, int n)   // n <= 64
    {
        if (n > 32) {
            put((uint32_t)v, 32);
            put((uint32_t)(v >> 32), n - 32);
        } else if (n > 0) {
            put((uint32_t)v, n);
        }
    }
    __device__ __forceinline__ int bits() const { return nw * 32 + nacc; }
    __device__ __forceinline__ int flush()
    {
        const int b = bits();
        if (nacc > 0) store((uint32_t)acc);
        return b;
    }
};

__device__ __forceinline__ unsigned long long low_mask(int n)
{
    return n >= 64 ? ~0ull : ((1ull << n) - 1ull);
}

// Row (lz, ly) of block bp (2D: row lz), the partial block's clamped samples
template <int DIMS>
__device__ __forceinline__ void load_row(const float* __restrict__ x, const CodecView& v, const BlockPos& bp,
                                         bool vec, int lz, int ly, float (&f)[4])
{
    const int xs = 4 * bp.bx;
    const int z = min(4 * bp.bz + lz, v.nz - 1);
    const int y = DIMS == 3 ? min(4 * bp.by + ly, v.ny - 1) : 0;
    const float* row = x + (long long)z * v.pz + (long long)y * v.py;
    if (vec) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(row + xs));
        f[0] = q.x; f[1] = q.y; f[2] = q.z; f[3] = q.w;
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) f[c] = __ldg(row + min(xs + c, v.nx - 1));
    }
}

// Raw form of a block: bits 1, 1, then the V float bit patterns, 32 bits
// each, LSB first; value i occupies bits 2 + 32 i .. 33 + 32 i, so word k
// holds the top two bits of value k-1 and the low 30 bits of value k.
// Words 0 .. V go to the block's stream area.
template <int DIMS>
__device__ __forceinline__ void raw_block(const float* __restrict__ x, const CodecView& v, const BlockPos& bp,
                                          uint32_t* __restrict__ gs)
{
    constexpr int ROWS = DIMS == 3 ? 16 : 4;
    uint32_t prev = 3u;      // the two header bits (as the "top bits" of value -1: 3 >> 30 would drop them)
    bool first = true;
#pragma unroll 1
    for (int r = 0; r < ROWS; ++r) {
        float f[4];
        load_row<DIMS>(x, v, bp, false, DIMS == 3 ? r / 4 : r, DIMS == 3 ? r % 4 : 0, f);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const uint32_t g = __float_as_uint(f[c]);
            gs[4 * r + c] = (first ? prev : (prev >> 30)) | (g << 2);
            first = false;
            prev = g;
        }
    }
    gs[Cfg<DIMS>::V] = prev >> 30;
}

// Shared-column offset of the coefficient of sequency rank R (a
// compile-time constant; ranks past V read row 0, never used)
template <int DIMS, int R>
__device__ __forceinline__ uint32_t at_rank(const uint32_t* col)
{
    constexpr int i = R < Cfg<DIMS>::V ? make_perm(DIMS).p[R < 64 ? R : 0] : 0;
    return R < Cfg<DIMS>::V ? col[i * ENC_THREADS] : 0u;
}
template <int DIMS, int H, int... R>
__device__ __forceinline__ void gather_ranks(uint32_t (&m)[32], const uint32_t* col, std::integer_sequence<int, R...>)
{
    ((m[R] = at_rank<DIMS, 32 * H + R>(col)), ...);
}

// Row of plane p of half h (see step 5 of encode_block)
__constant__ Perm c_perm3 = make_perm(3);
template <int DIMS> __device__ __forceinline__ int plane_row(int h, int p)
{
    return DIMS == 3 ? c_perm3.p[32 * h + p] : p;
}
template <int DIMS, int H, int R>
__device__ __forceinline__ void put_plane(uint32_t v, uint32_t* col)
{
    constexpr int row = DIMS == 3 ? make_perm(3).p[32 * H + R] : R;
    col[row * ENC_THREADS] = v;
}
template <int DIMS, int H, int... R>
__device__ __forceinline__ void scatter_planes(const uint32_t (&m)[32], uint32_t* col, std::integer_sequence<int, R...>)
{
    (put_plane<DIMS, H, R>(m[R], col), ...);
}

// Encode block b; returns its bit count, with the stream in gs (the block's
// area of the chunk's staging slot, 16-byte aligned).  The block is processed in
// four z slices (2D: four rows) so that only one slice's values are held in
// registers outside the closed-loop search, which keeps the code small and
// the register count low.  col is this thread's one column of shared memory
// (stride ENC_THREADS): the slice values, then the transformed coefficients
// (natural order, as negabinary), then the bit-plane words (step 5).  The
// closed loop's reference integers wait in gs until the stream overwrites
// them, so one shared column a thread suffices (half the shared memory of
// keeping them there too, twice the warps an SM holds).
template <int DIMS>
__device__ __forceinline__ int encode_block(const float* __restrict__ x, const CodecView& v, const Geo& G,
                                            float tol_f, long long b, uint32_t* col, uint32_t* __restrict__ gs,
                                            int* err)
{
    constexpr int V = Cfg<DIMS>::V;
    constexpr int SL = V / 4;                 // values per slice
    constexpr int S = ENC_THREADS;
    const BlockPos bp = block_pos(G, b);
    const bool vec = v.aligned && 4 * bp.bx + 3 < v.nx;
    // 1. finiteness and max |x| over the block's rows (the values are read
    // again, from the caches, in step 2)
    float amax = 0.0f;
    bool bad = false;
#pragma unroll
    for (int r = 0; r < V / 4; ++r) {
        float f[4];
        load_row<DIMS>(x, v, bp, vec, DIMS == 3 ? r / 4 : r, DIMS == 3 ? r % 4 : 0, f);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            bad |= !isfinite(f[c]);
            amax = fmaxf(amax, fabsf(f[c]));
        }
    }
    if (bad) atomicOr(err, 1);
    if (bad || amax <= tol_f) {
        gs[0] = 0u;                           // the single 0 bit
        return 1;
    }
    // block exponent: that of the largest magnitude (float order is exponent order)
    const int emax = max((int)(__float_as_uint(amax) >> 23), 1) - 127;
    // i = trunc(x 2^(23-Emax)): the scaling by a power of two is exact (the
    // product stays below 2^24; a product that underflows is below 1 and
    // truncates to 0 either way), so this equals the mantissa shift of the
    // definition
    const int sc = 23 - emax;
    const int sa = min(sc, 127);
    const float s1 = pow2f(sa), s2 = pow2f(sc - sa);
    // 2. integers (kept in the block's stream area for the closed loop), lifts along x and y
#pragma unroll 1
    for (int sl = 0; sl < 4; ++sl) {
        int32_t c[SL];
#pragma unroll
        for (int ly = 0; ly < SL / 4; ++ly) {
            float f[4];
            load_row<DIMS>(x, v, bp, vec, sl, ly, f);
#pragma unroll
            for (int q = 0; q < 4; ++q) c[4 * ly + q] = __float2int_rz(__fmul_rn(__fmul_rn(f[q], s1), s2));
        }
#pragma unroll
        for (int k = 0; k < SL; k += 4)        // the closed loop's reference
            *reinterpret_cast<int4*>(gs + SL * sl + k) = make_int4(c[k], c[k + 1], c[k + 2], c[k + 3]);
#pragma unroll
        for (int r = 0; r < SL / 4; ++r) lift_fwd(c[4 * r], c[4 * r + 1], c[4 * r + 2], c[4 * r + 3]);
        if constexpr (DIMS == 3) {
#pragma unroll
            for (int xx = 0; xx < 4; ++xx) lift_fwd(c[xx], c[4 + xx], c[8 + xx], c[12 + xx]);
        }
#pragma unroll
        for (int k = 0; k < SL; ++k) col[(SL * sl + k) * S] = (uint32_t)c[k];
    }
    // 3. lifts along z (across slices), negabinary
    uint32_t orall = 0;
#pragma unroll 1
    for (int k = 0; k < SL; ++k) {
        int32_t a0 = (int32_t)col[k * S], a1 = (int32_t)col[(SL + k) * S];
        int32_t a2 = (int32_t)col[(2 * SL + k) * S], a3 = (int32_t)col[(3 * SL + k) * S];
        lift_fwd(a0, a1, a2, a3);
        const uint32_t n0 = nega(a0), n1 = nega(a1), n2 = nega(a2), n3 = nega(a3);
        col[k * S] = n0;
        col[(SL + k) * S] = n1;
        col[(2 * SL + k) * S] = n2;
        col[(3 * SL + k) * S] = n3;
        orall |= n0 | n1 | n2 | n3;
    }
    const int ptop = orall ? 31 - __clz(orall) : 0;
    asm volatile("" ::: "memory");
    // 4. closed loop: the first plane whose truncation reproduces every integer within T - 2
    const float Tf = tol_f * pow2f(23 - emax);
    const int T = (int)Tf;
    int pbot = -1;
    if (T >= 2 && emax < 126) {
        const int lg = 31 - __clz(T);
        const int p0 = min(max(lg - GUARD, 0), ptop);
#pragma unroll 1
        for (int p = p0; p >= 0; --p) {
            const uint32_t mask = ~((1u << p) - 1u);
            int32_t t[V];
#pragma unroll
            for (int i = 0; i < V; ++i) t[i] = unnega(col[i * S] & mask);
            // the inverse transform's lifts along z first (they mix the
            // slices), then slice by slice the lifts within it and the
            // comparison (the lifts are those of xform_inv, in an order that
            // changes no result; leaving at the first failing slice was
            // slower: the branch costs spills)
            if constexpr (DIMS == 3) {
#pragma unroll
                for (int r = 0; r < 16; ++r) lift_inv(t[r], t[16 + r], t[32 + r], t[48 + r]);
            } else {
#pragma unroll
                for (int xx = 0; xx < 4; ++xx) lift_inv(t[xx], t[4 + xx], t[8 + xx], t[12 + xx]);
            }
            // |i - t| <= T - 2 as one unsigned comparison (|i|, |t| < 2^26,
            // T <= 2^24 because max|x| > tol)
            const uint32_t lim = (uint32_t)(T - 2);
            bool ok = true;
#pragma unroll
            for (int sl = 0; sl < 4; ++sl) {
                int32_t* u = t + SL * sl;
                if constexpr (DIMS == 3) {
#pragma unroll
                    for (int xx = 0; xx < 4; ++xx) lift_inv(u[xx], u[4 + xx], u[8 + xx], u[12 + xx]);
#pragma unroll
                    for (int r = 0; r < 4; ++r) lift_inv(u[4 * r], u[4 * r + 1], u[4 * r + 2], u[4 * r + 3]);
                } else {
                    lift_inv(u[0], u[1], u[2], u[3]);
                }
                // the reference loads of one slice at a time, after its lifts
                asm volatile("" ::: "memory");
#pragma unroll
                for (int k = 0; k < SL; k += 4) {
                    const int4 r = *reinterpret_cast<const int4*>(gs + SL * sl + k);
                    ok &= (uint32_t)(r.x - u[k]) + lim <= 2u * lim;
                    ok &= (uint32_t)(r.y - u[k + 1]) + lim <= 2u * lim;
                    ok &= (uint32_t)(r.z - u[k + 2]) + lim <= 2u * lim;
                    ok &= (uint32_t)(r.w - u[k + 3]) + lim <= 2u * lim;
                }
            }
            if (ok) {
                pbot = p;
                break;
            }
        }
    }
    if (pbot >= 0) {
        // 5. bit-plane words: sequency-ordered coefficients, transposed 32 at
        // a time.  3D: plane p of half h goes to the row of the coefficient
        // of rank 32 h + p (free once its half has been read, and never an
        // input of the other half); 2D: the one half's plane p to row p.
        asm volatile("" ::: "memory");
        {
            uint32_t m[32];
            gather_ranks<DIMS, 0>(m, col, std::make_integer_sequence<int, 32>{});
            transpose32(m);
            scatter_planes<DIMS, 0>(m, col, std::make_integer_sequence<int, 32>{});
        }
        if constexpr (V > 32) {
            uint32_t m[32];
            gather_ranks<DIMS, 1>(m, col, std::make_integer_sequence<int, 32>{});
            transpose32(m);
            scatter_planes<DIMS, 1>(m, col, std::make_integer_sequence<int, 32>{});
        }
        // 6. the stream, into the block's area of the staging slot
        asm volatile("" ::: "memory");
        BitW<DIMS> bw{gs, 0ull, 0, 0};
        bw.put(1u | ((uint32_t)(emax + 127) << 2) | ((uint32_t)ptop << 10) | ((uint32_t)pbot << 15), 20);
        int s = 0;
#pragma unroll 1
        for (int p = ptop; p >= pbot; --p) {
            unsigned long long W = col[plane_row<DIMS>(0, p) * S];
            if (V > 32) W |= (unsigned long long)col[plane_row<DIMS>(1, p) * S] << 32;
            bw.put64(W & low_mask(s), s);
            while (s < V) {
                const unsigned long long rest = s < 64 ? W >> s : 0ull;
                if (rest == 0ull) {
                    bw.put(0u, 1);
                    break;
                }
                const int z = __ffsll((long long)rest) - 1;
                // a group test (1), z zeros, the set bit (1)
                if (z <= 29) {
                    bw.put(1u | (2u << z), z + 2);
                } else {
                    bw.put(1u, 1);
                    bw.put64(1ull << z, z + 1);
                }
                s += z + 1;
            }
            if (bw.nw > V) break;             // longer than raw already
        }
        if (bw.bits() <= Cfg<DIMS>::MAXBITS) return bw.flush();
        // longer than raw: the raw form replaces it
    }
    raw_block<DIMS>(x, v, bp, gs);
    return Cfg<DIMS>::MAXBITS;
}

// One thread per block; each warp owns one 32-block chunk.  After its
// blocks are coded (each into its own area of the chunk's staging slot),
// the warp assembles the chunk's bits contiguously in its part of the
// shared columns (plus two words of xtra), writes them back over the
// staging slot, writes its word count, and adds the count to the sums of
// its groups of 32 and of 1024 chunks (the compaction's offsets).
constexpr int ENC_MIN_CTAS = 10;
template <int DIMS>
__global__ void __launch_bounds__(ENC_THREADS, ENC_MIN_CTAS) enc_kernel(const float* __restrict__ x, CodecView v,
                                                          Geo G, float tol_f, uint32_t* __restrict__ scratch,
                                                          uint32_t* __restrict__ out, const long long* base_word,
                                                          long long cap_words, int* err)
{
    constexpr int V = Cfg<DIMS>::V;
    constexpr int CWD = V > 32 ? V : 32;       // plane words need 32 rows even in 2D
    constexpr int S = ENC_THREADS;
    constexpr int MW = Cfg<DIMS>::AREA;
    __shared__ uint32_t colw[CWD * ENC_THREADS];
    __shared__ uint32_t xtra[ENC_THREADS / 32][4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long b = (long long)blockIdx.x * ENC_THREADS + threadIdx.x;
    const long long base = *base_word;
    if (base + G.table_words > cap_words) {
        if (b == 0) atomicOr(err, 2);
        return;
    }
    const ScratchLayout L = scratch_layout(G);
    uint16_t* sizes = reinterpret_cast<uint16_t*>(out + base + HDR + G.nchunks);
    if (b == 0 && (G.nblocks & 1)) sizes[G.nblocks] = 0;
    const long long c = b / CHUNK;
    uint32_t* stage = scratch + L.stage + c * L.cw;          // dereferenced only for c < nchunks
    uint32_t* gs = stage + (b % CHUNK) * MW;
    int nbits = 0;
    if (b < G.nblocks) {
        nbits = encode_block<DIMS>(x, v, G, tol_f, b, colw + threadIdx.x, gs, err);
        sizes[b] = (uint16_t)nbits;
    }
    if (c >= G.nchunks) return;                // whole warp
    __syncwarp();
    int incl = nbits;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const int totb = __shfl_sync(0xffffffffu, incl, 31);
    const int off = incl - nbits;
    const int words = (totb + 31) / 32;
    // word j of the chunk: row j / 32, this warp's column j % 32 of the
    // shared columns (32 CWD words), then xtra
    uint32_t* sv = colw + 32 * wid;
    auto bufw = [&](int j) -> uint32_t* { return j < 32 * CWD ? sv + (j >> 5) * S + (j & 31) : &xtra[wid][j - 32 * CWD]; };
    for (int k = lane; k < words; k += 32) *bufw(k) = 0u;
    __syncwarp();
    const int sw = (nbits + 31) / 32;
    for (int k = 0; k < sw; ++k) {
        uint32_t val = gs[k];
        const int rem = nbits - 32 * k;
        if (rem < 32) val &= (1u << rem) - 1u;
        const int pos = off + 32 * k;
        const int sh = pos & 31, idx = pos >> 5;
        atomicOr(bufw(idx), val << sh);
        if (sh) atomicOr(bufw(idx + 1), val >> (32 - sh));
    }
    // every block's stream has been read: the slot takes the assembled chunk
    __syncwarp();
    for (int k = lane; k < words; k += 32) stage[k] = *bufw(k);
    if (lane == 0) {
        scratch[L.counts + c] = (uint32_t)words;
        atomicAdd(scratch + L.g1 + (c >> 5), (uint32_t)words);
        atomicAdd(scratch + L.g2 + (c >> 10), (uint32_t)words);
    }
}

// Compaction: a 128-thread CTA moves CPB consecutive chunks from their
// staging slots to the payload.  Its payload offset is the sum of the whole
// groups of 1024 chunks before it, of the groups of 32 before it inside its
// group of 1024, and of the chunks before it inside its group of 32 (at most
// chunks / 1024 + 62 values, all loaded at once; linear total work).  The
// sums of the groups of 1024 also give the stream's total, which decides the
// overflow (nothing is written) and, in CTA 0, the header, the pool's next
// word and the statistics.  The last CTA to finish reading the sums (a
// counter, no waiting) sets them back to zero for the next compression.
// Small CTAs spread the copy over every SM.
constexpr int CMP_THREADS = 128;
constexpr int CPB = 4;

template <int DIMS>
__global__ void __launch_bounds__(CMP_THREADS) compact_kernel(uint32_t* __restrict__ out, const long long* base_word,
                                                              long long cap_words, long long* next_word, Geo G,
                                                              float tol_f, uint32_t* __restrict__ scratch,
                                                              int* err, unsigned long long* stat_words)
{
    constexpr int NW = CMP_THREADS / 32;
    __shared__ long long red[2][NW];
    __shared__ uint32_t offs[CPB + 1];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long base = *base_word;
    if (base + G.table_words > cap_words) {            // the encoder raised the error
        if (blockIdx.x == 0 && threadIdx.x == 0) *next_word = base;
        return;
    }
    const ScratchLayout L = scratch_layout(G);
    const long long ng1 = (G.nchunks + 31) / 32, ng2 = (G.nchunks + 1023) / 1024;
    const uint32_t* counts = scratch + L.counts;
    uint32_t* g1 = scratch + L.g1;
    uint32_t* g2 = scratch + L.g2;
    const long long c0 = (long long)blockIdx.x * CPB;
    const long long q2 = c0 >> 10, q1 = c0 >> 5;
    long long before = 0, total = 0;
    for (long long i = threadIdx.x; i < ng2; i += CMP_THREADS) {
        const uint32_t w = g2[i];
        total += w;
        if (i < q2) before += w;
    }
    for (long long g = (q2 << 5) + threadIdx.x; g < q1; g += CMP_THREADS) before += g1[g];
    for (long long k = (q1 << 5) + threadIdx.x; k < c0; k += CMP_THREADS) before += counts[k];
    if (threadIdx.x == 0) {                            // offsets of this CTA's chunks
        uint32_t o = 0;
        for (int k = 0; k < CPB; ++k) {
            offs[k] = o;
            if (c0 + k < G.nchunks) o += counts[c0 + k];
        }
        offs[CPB] = o;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        before += __shfl_xor_sync(0xffffffffu, before, o);
        total += __shfl_xor_sync(0xffffffffu, total, o);
    }
    if (lane == 0) {
        red[0][wid] = before;
        red[1][wid] = total;
    }
    __syncthreads();
    long long prefix = 0;
    total = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        prefix += red[0][k];
        total += red[1][k];
    }
    // every thread of this CTA has read the sums; the last CTA resets them
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(scratch, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (long long i = threadIdx.x; i < ng1; i += CMP_THREADS) g1[i] = 0u;
        for (long long i = threadIdx.x; i < ng2; i += CMP_THREADS) g2[i] = 0u;
        if (threadIdx.x == 0) scratch[0] = 0u;
    }
    const long long end = base + G.table_words + total;
    uint32_t* hdr = out + base;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        hdr[0] = MAGIC;
        hdr[1] = (uint32_t)G.dims | (VERSION << 8);
        hdr[2] = (uint32_t)G.nz;
        hdr[3] = (uint32_t)G.ny;
        hdr[4] = (uint32_t)G.nx;
        hdr[5] = (uint32_t)G.nblocks;
        hdr[6] = (uint32_t)G.nchunks;
        hdr[7] = (uint32_t)total;
        hdr[8] = __float_as_uint(tol_f);
        hdr[9] = (*err & 1) ? 1u : 0u;
        for (int i = 10; i < HDR; ++i) hdr[i] = 0u;
        if (end > cap_words) {
            atomicOr(err, 2);
            *next_word = base;
        } else {
            *next_word = end;
        }
        if (stat_words) atomicAdd(stat_words, (unsigned long long)(G.table_words + total));
    }
    if (end > cap_words) return;                       // overflow: nothing is written
    if (threadIdx.x < CPB && c0 + threadIdx.x < G.nchunks) {
        const int k = threadIdx.x;
        if (offs[k + 1] - offs[k] > (uint32_t)L.cw) atomicOr(err, 4);   // not a count the encoder can write
        hdr[HDR + c0 + k] = (uint32_t)(prefix + offs[k]);
    }
    // the CTA's chunks are contiguous in the payload: every thread copies
    // words of them (all loads independent, so their latencies overlap)
    const uint32_t gw = offs[CPB];
    uint32_t* payload = out + base + G.table_words + prefix;
    const uint32_t* stage = scratch + L.stage + c0 * L.cw;
    for (uint32_t w = threadIdx.x; w < gw; w += CMP_THREADS) {
        int lo = 0;
#pragma unroll
        for (int k = 1; k < CPB; ++k)
            if (offs[k] <= w) lo = k;
        payload[w] = stage[(long long)lo * L.cw + (w - offs[lo])];
    }
}

// 64 stream bits starting at bit `pos` of the payload (zeros past `limit` words)
__device__ __forceinline__ unsigned long long peek64(const uint32_t* __restrict__ p, long long pos, long long limit)
{
    const long long w = pos >> 5;
    const int sh = (int)(pos & 31);
    const unsigned long long w0 = w < limit ? p[w] : 0u;
    const unsigned long long w1 = w + 1 < limit ? p[w + 1] : 0u;
    const unsigned long long w2 = w + 2 < limit ? p[w + 2] : 0u;
    unsigned long long v = (w0 | (w1 << 32)) >> sh;
    if (sh) v |= w2 << (64 - sh);
    return v;
}

template <int DIMS>
__global__ void __launch_bounds__(DEC_THREADS, 5) dec_kernel(const uint32_t* __restrict__ in, const long long* base_word,
                                                          long long cap_words, Geo G, CodecView v,
                                                          float* __restrict__ x, int* err)
{
    constexpr int V = Cfg<DIMS>::V;
    constexpr int CWD = V > 32 ? V : 32;
    __shared__ uint32_t colw[CWD * DEC_THREADS];
    uint32_t* col = colw + threadIdx.x;
    const long long b = (long long)blockIdx.x * DEC_THREADS + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const long long c = b / CHUNK;
    if (c >= G.nchunks) return;                    // whole warp
    const long long base = *base_word;
    if (base < 0 || base + G.table_words > cap_words) {
        if (lane == 0) atomicOr(err, 4);
        return;
    }
    const uint32_t* hdr = in + base;
    if (hdr[0] != MAGIC || hdr[1] != ((uint32_t)G.dims | (VERSION << 8)) || hdr[2] != (uint32_t)G.nz ||
        hdr[3] != (uint32_t)G.ny || hdr[4] != (uint32_t)G.nx || hdr[5] != (uint32_t)G.nblocks ||
        hdr[6] != (uint32_t)G.nchunks || base + G.table_words + (long long)hdr[7] > cap_words) {
        if (lane == 0) atomicOr(err, 4);
        return;
    }
    const long long pw = hdr[7];
    const uint32_t* payload = hdr + G.table_words;
    const uint16_t* sizes = reinterpret_cast<const uint16_t*>(hdr + HDR + G.nchunks);
    const bool valid = b < G.nblocks;
    const int nbits = valid ? sizes[b] : 0;
    int incl = nbits;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (!valid) return;
    const long long start = (long long)hdr[HDR + c] * 32 + (incl - nbits);
    const long long end = start + nbits;
    if (end > pw * 32) {
        atomicOr(err, 4);
        return;
    }
    long long pos = start;
    bool corrupt = false;
    float f[V];
    const unsigned long long h0 = peek64(payload, pos, pw);
    if (!(h0 & 1ull)) {
        pos += 1;
#pragma unroll
        for (int i = 0; i < V; ++i) f[i] = 0.0f;
    } else if (h0 & 2ull) {
        pos += 2;
#pragma unroll
        for (int i = 0; i < V; ++i) {
            f[i] = __uint_as_float((uint32_t)peek64(payload, pos, pw));
            pos += 32;
        }
    } else {
        const int emax = (int)((h0 >> 2) & 0xFFu) - 127;
        const int ptop = (int)((h0 >> 10) & 31u);
        const int pbot = (int)((h0 >> 15) & 31u);
        pos += 20;
        if (emax < -126 || emax > 127 || pbot > ptop) corrupt = true;
        // plane words into this thread's shared column (rows p and 32 + p),
        // then one bit-matrix transpose gives the coefficient words
        constexpr int S = DEC_THREADS;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            col[q * S] = 0u;
            if (V > 32) col[(32 + q) * S] = 0u;
        }
        int s = 0;
#pragma unroll 1
        for (int p = ptop; p >= pbot && !corrupt; --p) {
            unsigned long long W = 0;
            if (s > 0) {
                W = peek64(payload, pos, pw) & low_mask(s);
                pos += s;
            }
            while (s < V) {
                // one look at the group test and the run after it; a run
                // longer than the 63 bits past the test takes a second look
                const unsigned long long t = peek64(payload, pos, pw);
                if (!(t & 1ull)) {
                    pos += 1;
                    break;
                }
                unsigned long long look = t >> 1;
                int z;
                if (look != 0ull) {
                    z = __ffsll((long long)look) - 1;
                } else {
                    look = peek64(payload, pos + 1, pw);
                    if (look == 0ull) { corrupt = true; break; }
                    z = __ffsll((long long)look) - 1;
                }
                if (s + z >= V) { corrupt = true; break; }
                W |= 1ull << (s + z);
                pos += z + 2;
                s += z + 1;
            }
            if (pos > end) corrupt = true;
            col[p * S] = (uint32_t)W;
            if (V > 32) col[(32 + p) * S] = (uint32_t)(W >> 32);
        }
#pragma unroll
        for (int h = 0; h < (V + 31) / 32; ++h) {
            uint32_t m[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) m[q] = col[(32 * h + q) * S];
            transpose32(m);
#pragma unroll
            for (int r = 0; r < 32; ++r) col[(32 * h + r) * S] = m[r];
        }
        asm volatile("" ::: "memory");
        int32_t t[V];
#pragma unroll
        for (int i = 0; i < V; ++i) t[i] = unnega(col[rank_of<DIMS>(i) * S]);
        xform_inv<DIMS>(t);
        const float sc = pow2f(max(emax - 23, -126));
#pragma unroll
        for (int i = 0; i < V; ++i) f[i] = __fmul_rn(__int2float_rn(t[i]), sc);
    }
    if (corrupt || pos != end) {
        atomicOr(err, 4);
        return;
    }
    // scatter the valid part of the block
    const BlockPos bp = block_pos(G, b);
    const int xs = 4 * bp.bx;
    const bool vec = v.aligned && xs + 3 < v.nx;
    constexpr int ROWS = DIMS == 3 ? 16 : 4;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const int z = 4 * bp.bz + (DIMS == 3 ? r / 4 : r);
        const int y = DIMS == 3 ? 4 * bp.by + r % 4 : 0;
        if (z >= v.nz || y >= v.ny) continue;
        float* row = x + (long long)z * v.pz + (long long)y * v.py;
        if (vec) {
            *reinterpret_cast<float4*>(row + xs) = make_float4(f[4 * r], f[4 * r + 1], f[4 * r + 2], f[4 * r + 3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (xs + q < v.nx) row[xs + q] = f[4 * r + q];
        }
    }
}

}  // namespace

long long codec_bound_words(int dims, int nz, int ny, int nx)
{
    const Geo G = make_geo(dims, nz, ny, nx);
    const long long per_chunk = dims == 3 ? (CHUNK * Cfg<3>::MAXBITS + 31) / 32 : (CHUNK * Cfg<2>::MAXBITS + 31) / 32;
    return G.table_words + G.nchunks * per_chunk;
}

long long codec_scratch_bytes(int dims, int nz, int ny, int nx)
{
    return scratch_layout(make_geo(dims, nz, ny, nx)).words * 4;
}

long long codec_scratch_zero_bytes(int dims, int nz, int ny, int nx)
{
    return scratch_zero_words(make_geo(dims, nz, ny, nx)) * 4;
}

cudaError_t codec_compress_dev(const float* x, const CodecView& v, float tol_f, uint32_t* out,
                               const long long* base_word, long long cap_words, long long* next_word,
                               void* scratch, int* err, unsigned long long* stat_words, cudaStream_t s)
{
    const Geo G = make_geo(v.dims, v.nz, v.ny, v.nx);
    uint32_t* sc = static_cast<uint32_t*>(scratch);
    const unsigned eb = (unsigned)((G.nblocks + ENC_THREADS - 1) / ENC_THREADS);
    const unsigned cb = (unsigned)((G.nchunks + CPB - 1) / CPB);
    if (v.dims == 3) {
        enc_kernel<3><<<eb, ENC_THREADS, 0, s>>>(x, v, G, tol_f, sc, out, base_word, cap_words, err);
        compact_kernel<3><<<cb, CMP_THREADS, 0, s>>>(out, base_word, cap_words, next_word, G, tol_f, sc, err,
                                                         stat_words);
    } else {
        enc_kernel<2><<<eb, ENC_THREADS, 0, s>>>(x, v, G, tol_f, sc, out, base_word, cap_words, err);
        compact_kernel<2><<<cb, CMP_THREADS, 0, s>>>(out, base_word, cap_words, next_word, G, tol_f, sc, err,
                                                         stat_words);
    }
    return cudaGetLastError();
}

cudaError_t codec_decompress_dev(const uint32_t* in, const long long* base_word, long long cap_words,
                                 const CodecView& v, float* x, int* err, cudaStream_t s)
{
    const Geo G = make_geo(v.dims, v.nz, v.ny, v.nx);
    const unsigned db = (unsigned)((G.nchunks * CHUNK + DEC_THREADS - 1) / DEC_THREADS);
    if (v.dims == 3)
        dec_kernel<3><<<db, DEC_THREADS, 0, s>>>(in, base_word, cap_words, G, v, x, err);
    else
        dec_kernel<2><<<db, DEC_THREADS, 0, s>>>(in, base_word, cap_words, G, v, x, err);
    return cudaGetLastError();
}

}  // namespace ckfwi
