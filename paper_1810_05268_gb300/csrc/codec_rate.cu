// Fixed-rate mode of the block codec (Sec. 2.2 lists ZFP's fixed-rate mode
// beside the fixed-tolerance one: a guaranteed size, no error bound).
//
//  rate     R bits per value, 1 <= R <= 32; every block occupies exactly
//           W = ceil(R 4^d / 32) words, a budget of 32 W bits, so a field
//           takes 16 + nblocks W words whatever its values.
//  block    0: all values +-0, a non-finite value (flag NONFINITE) or
//           Emax < -100 (values below 2^-99 are flushed); rest of the
//           budget zero.  Else 1, Emax+127 (8), ptop (5), then planes ptop
//           down to 0 coded as in the fixed-accuracy mode (verbatim bits of
//           the s significant coefficients, then group tests) until the
//           budget is full: the first bit that does not fit is dropped and
//           coding stops.  Integers, lifting, order and negabinary are the
//           fixed-accuracy mode's (codec_common.cuh).
//  decode   the same bits up to the budget; bits not read are zero;
//           x_hat = float(i_hat) 2^(Emax-23).
//  container header words of the fixed-accuracy mode with version 2,
//           [7] = nblocks W, [8] = R; the blocks back to back after it.
//
// GPU layout: one thread per block, as in the fixed-accuracy kernels.  The
// block's values live in registers (lifting, order and negabinary with
// compile-time indices); two 32 x 32 bit transposes turn the 64 coefficient
// words into 32 plane masks of 64 bits, kept in shared memory so that the
// coder can walk the planes with a run-time index.  On a 64-bit plane mask
// the verbatim bits are one masked append and a group test plus its run is
// one find-first-set.  The decoder parses the planes into the same masks
// and transposes them back.  No size table and no scan: block b sits at
// word 16 + b W of the stream.
#include "codec_common.cuh"

namespace ckfwi {
namespace {

constexpr uint32_t RATE_VERSION = 2u;
constexpr int RATE_EMIN = -100;
constexpr int RT = 64;                 // threads (blocks) per CTA

__host__ __device__ inline long long rate_block_words(int dims, int rate) { return ((long long)rate * (dims == 3 ? 64 : 16) + 31) / 32; }

__device__ __forceinline__ unsigned long long lowbits(int n) { return n >= 64 ? ~0ull : ((1ull << n) - 1ull); }

// Bit writer with a budget straight into the block's words: appends the
// low n bits of v while they fit; `full` once a bit was dropped.
struct RateW {
    uint32_t* o;
    unsigned long long acc;
    int nacc, nw, left;
    bool full;
    __device__ __forceinline__ void put(unsigned long long v, int n)   // n <= 64
    {
        if (full || n <= 0) return;
        if (n > left) {
            n = left;
            full = true;
        }
        left -= n;
        while (n > 0) {
            const int k = min(n, 32);
            acc |= (v & lowbits(k)) << nacc;
            nacc += k;
            v = k == 64 ? 0 : (v >> k);
            n -= k;
            if (nacc >= 32) {
                o[nw++] = (uint32_t)acc;
                acc >>= 32;
                nacc -= 32;
            }
        }
    }
    __device__ __forceinline__ void finish(int W)   // the partial word, then zeros to the budget
    {
        if (nacc > 0) o[nw++] = (uint32_t)acc;
        for (; nw < W; ++nw) o[nw] = 0u;
    }
};

__global__ void rate_header_kernel(uint32_t* __restrict__ out, const long long* base_word, long long cap_words,
                                   long long* next_word, Geo G, int rate, int* err, unsigned long long* stat_words)
{
    const long long W = rate_block_words(G.dims, rate);
    const long long total = HDR + G.nblocks * W;
    const long long base = *base_word;
    if (base + total > cap_words) {
        if (threadIdx.x == 0) {
            atomicOr(err, 2);
            *next_word = base;
        }
        return;
    }
    uint32_t* o = out + base;
    if (threadIdx.x < HDR) {
        uint32_t h = 0;
        switch (threadIdx.x) {
        case 0: h = MAGIC; break;
        case 1: h = (uint32_t)G.dims | (RATE_VERSION << 8); break;
        case 2: h = (uint32_t)G.nz; break;
        case 3: h = (uint32_t)G.ny; break;
        case 4: h = (uint32_t)G.nx; break;
        case 5: h = (uint32_t)G.nblocks; break;
        case 7: h = (uint32_t)(G.nblocks * W); break;
        case 8: h = (uint32_t)rate; break;
        default: h = 0;
        }
        o[threadIdx.x] = h;
    }
    if (threadIdx.x == 0) {
        *next_word = base + total;
        if (stat_words) *stat_words = (unsigned long long)total;
    }
}

template <int DIMS>
__global__ void __launch_bounds__(RT) rate_enc_kernel(const float* __restrict__ x, CodecView v, Geo G, int rate,
                                                      uint32_t* __restrict__ out, const long long* base_word,
                                                      long long cap_words, int* err)
{
    constexpr int V = Cfg<DIMS>::V;
    constexpr Perm P = make_perm(DIMS);
    __shared__ unsigned long long spl[32][RT];      // plane masks of each thread's block
    const int tid = threadIdx.x;
    const long long b = (long long)blockIdx.x * RT + tid;
    if (b >= G.nblocks) return;
    const int W = (int)rate_block_words(DIMS, rate);
    const long long base = *base_word;
    if (base + HDR + G.nblocks * W > cap_words) return;     // the header kernel raised the error
    uint32_t* o = out + base + HDR + b * W;

    float f[V];
    gather<DIMS>(x, v, block_pos(G, b), f);
    bool bad = false;
    int emax = -1000;
#pragma unroll
    for (int i = 0; i < V; ++i) {
        const uint32_t u = __float_as_uint(f[i]);
        bad = bad || !isfinite(f[i]);
        const int be = (int)((u >> 23) & 0xFF);
        if ((u & 0x7FFFFFFFu) != 0) emax = max(emax, (be > 0 ? be : 1) - 127);
    }
    if (bad || emax < RATE_EMIN) {           // zero-coded block (no non-zero value: emax = -1000)
        if (bad) {
            atomicOr(err, 1);
            atomicOr(out + base + 9, 1u);
        }
        for (int k = 0; k < W; ++k) o[k] = 0u;
        return;
    }
    int32_t iv[V];
#pragma unroll
    for (int i = 0; i < V; ++i) {
        const uint32_t u = __float_as_uint(f[i]);
        const int be = (int)((u >> 23) & 0xFF);
        const uint32_t M = (u & 0x7FFFFFu) | (be > 0 ? 0x800000u : 0u);
        const int sh = emax - ((be > 0 ? be : 1) - 127);
        uint32_t mag = sh >= 32 ? 0u : (M >> sh);
        if ((u & 0x7FFFFFFFu) == 0) mag = 0;
        iv[i] = (u >> 31) ? -(int32_t)mag : (int32_t)mag;
    }
    xform_fwd<DIMS>(iv);
    uint32_t lo[32], hi[32], orall = 0;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        lo[r] = r < V ? nega(iv[P.p[r]]) : 0u;
        hi[r] = r + 32 < V ? nega(iv[P.p[r + 32 < V ? r + 32 : 0]]) : 0u;
        orall |= lo[r] | hi[r];
    }
    const int ptop = orall ? 31 - __clz(orall) : 0;
    transpose32(lo);
    if (V > 32) transpose32(hi);
#pragma unroll
    for (int p = 0; p < 32; ++p) spl[p][tid] = (unsigned long long)lo[p] | ((unsigned long long)hi[p] << 32);

    RateW wr{o, 0ull, 0, 0, 32 * W, false};
    wr.put(1u, 1);
    wr.put((unsigned long long)(emax + 127), 8);
    wr.put((unsigned long long)ptop, 5);
    int sgn = 0;   // coefficients already significant
    for (int p = ptop; p >= 0 && !wr.full; --p) {
        const unsigned long long m = spl[p][tid];
        wr.put(m & lowbits(sgn), sgn);
        while (!wr.full && sgn < V) {
            const unsigned long long rest = m >> sgn;
            wr.put(rest ? 1u : 0u, 1);
            if (!rest || wr.full) break;
            const int fz = __ffsll((long long)rest) - 1;   // zeros before the next significant one
            wr.put(1ull << fz, fz + 1);
            sgn += fz + 1;
        }
    }
    wr.finish(W);
}

// Bit reader over a block's words in global memory, with the same budget.
struct RateR {
    const uint32_t* w;
    int pos, end, nwd;
    bool more;
    __device__ __forceinline__ unsigned long long peek64() const   // 64 bits from pos, zeros past the end
    {
        const int k = pos >> 5, sh = pos & 31;
        const unsigned long long a = k < nwd ? __ldg(w + k) : 0u, b = k + 1 < nwd ? __ldg(w + k + 1) : 0u,
                                 c = k + 2 < nwd ? __ldg(w + k + 2) : 0u;
        unsigned long long r = (a | (b << 32)) >> sh;
        if (sh) r |= c << (64 - sh);
        return r;
    }
    __device__ __forceinline__ unsigned long long get(int n)   // n <= 64; stops when the budget runs out
    {
        if (!more) return 0;
        if (n > end - pos) {
            more = false;
            return 0;
        }
        const unsigned long long r = peek64() & lowbits(n);
        pos += n;
        return r;
    }
};

template <int DIMS>
__global__ void __launch_bounds__(RT) rate_dec_kernel(const uint32_t* __restrict__ in, const long long* base_word,
                                                      long long cap_words, Geo G, int rate, CodecView v,
                                                      float* __restrict__ x, int* err)
{
    constexpr int V = Cfg<DIMS>::V;
    constexpr Perm P = make_perm(DIMS);
    __shared__ unsigned long long spl[32][RT];
    const int tid = threadIdx.x;
    const long long b = (long long)blockIdx.x * RT + tid;
    if (b >= G.nblocks) return;
    const int W = (int)rate_block_words(DIMS, rate);
    const long long base = *base_word;
    if (base < 0 || base + HDR + G.nblocks * W > cap_words) {
        atomicOr(err, 4);
        return;
    }
    const uint32_t* h = in + base;
    if (__ldg(h) != MAGIC || __ldg(h + 1) != ((uint32_t)DIMS | (RATE_VERSION << 8)) || __ldg(h + 2) != (uint32_t)G.nz ||
        __ldg(h + 3) != (uint32_t)G.ny || __ldg(h + 4) != (uint32_t)G.nx || __ldg(h + 5) != (uint32_t)G.nblocks ||
        __ldg(h + 7) != (uint32_t)(G.nblocks * W) || __ldg(h + 8) != (uint32_t)rate) {
        atomicOr(err, 4);
        return;
    }
    RateR rd{h + HDR + b * W, 0, 32 * W, W, true};
    float f[V];
    const bool coded = rd.get(1) != 0;
    if (!coded) {
#pragma unroll
        for (int i = 0; i < V; ++i) f[i] = 0.0f;
    } else {
        const int emax = (int)rd.get(8) - 127;
        const int ptop = (int)rd.get(5);
#pragma unroll
        for (int p = 0; p < 32; ++p) spl[p][tid] = 0ull;
        int sgn = 0;
        for (int p = ptop; p >= 0 && rd.more; --p) {
            // verbatim bits of the significant coefficients (as many as the budget holds)
            const int k = min(sgn, rd.end - rd.pos);
            unsigned long long m = rd.get(k);
            if (k < sgn) rd.more = false;
            while (rd.more && sgn < V) {
                const unsigned long long g = rd.get(1);
                if (!rd.more || !g) break;
                // coefficients sgn, sgn+1, ... up to and including the first set one
                const int avail = min(V - sgn, rd.end - rd.pos);
                const unsigned long long win = rd.peek64() & lowbits(avail);
                if (win) {
                    const int fz = __ffsll((long long)win) - 1;
                    m |= 1ull << (sgn + fz);
                    rd.pos += fz + 1;
                    sgn += fz + 1;
                } else {
                    rd.pos += avail;
                    sgn += avail;
                    if (sgn < V) rd.more = false;   // the budget ended inside the run
                }
            }
            spl[p][tid] = m;
        }
        uint32_t lo[32], hi[32];
#pragma unroll
        for (int p = 0; p < 32; ++p) {
            const unsigned long long m = spl[p][tid];
            lo[p] = (uint32_t)m;
            hi[p] = (uint32_t)(m >> 32);
        }
        transpose32(lo);
        if (V > 32) transpose32(hi);
        int32_t iv[V];
#pragma unroll
        for (int r = 0; r < V; ++r) iv[P.p[r]] = unnega(r < 32 ? lo[r] : hi[r < 32 ? 0 : r - 32]);
        xform_inv<DIMS>(iv);
        const float sc = pow2f(max(emax - 23, -126));
#pragma unroll
        for (int i = 0; i < V; ++i) f[i] = __fmul_rn(__int2float_rn(iv[i]), sc);
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

long long codec_rate_words(int dims, int nz, int ny, int nx, int rate)
{
    if (rate < 1 || rate > 32) return -1;
    const Geo G = make_geo(dims, nz, ny, nx);
    return HDR + G.nblocks * rate_block_words(dims, rate);
}

cudaError_t codec_rate_compress_dev(const float* x, const CodecView& v, int rate, uint32_t* out,
                                    const long long* base_word, long long cap_words, long long* next_word, int* err,
                                    unsigned long long* stat_words, cudaStream_t s)
{
    if (rate < 1 || rate > 32) return cudaErrorInvalidValue;
    const Geo G = make_geo(v.dims, v.nz, v.ny, v.nx);
    const unsigned nb = (unsigned)((G.nblocks + RT - 1) / RT);
    rate_header_kernel<<<1, 32, 0, s>>>(out, base_word, cap_words, next_word, G, rate, err, stat_words);
    if (v.dims == 3) rate_enc_kernel<3><<<nb, RT, 0, s>>>(x, v, G, rate, out, base_word, cap_words, err);
    else rate_enc_kernel<2><<<nb, RT, 0, s>>>(x, v, G, rate, out, base_word, cap_words, err);
    return cudaGetLastError();
}

cudaError_t codec_rate_decompress_dev(const uint32_t* in, const long long* base_word, long long cap_words,
                                      const CodecView& v, int rate, float* x, int* err, cudaStream_t s)
{
    if (rate < 1 || rate > 32) return cudaErrorInvalidValue;
    const Geo G = make_geo(v.dims, v.nz, v.ny, v.nx);
    const unsigned nb = (unsigned)((G.nblocks + RT - 1) / RT);
    if (v.dims == 3) rate_dec_kernel<3><<<nb, RT, 0, s>>>(in, base_word, cap_words, G, rate, v, x, err);
    else rate_dec_kernel<2><<<nb, RT, 0, s>>>(in, base_word, cap_words, G, rate, v, x, err);
    return cudaGetLastError();
}

}  // namespace ckfwi
