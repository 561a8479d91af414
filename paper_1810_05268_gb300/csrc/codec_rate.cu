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
// GPU layout: one warp per block.  Lane l holds values / coefficients l and
// l + 32; the lifting runs in the warp's shared scratch; each plane's
// significance bits come from two ballots, so the coder works on a 64-bit
// plane mask: verbatim bits are one masked append, a group test and the run
// up to the next significant coefficient one find-first-set.  Every lane
// runs the same (uniform) coder state; the words go through shared memory
// and are stored by the warp together.  No size table, no scan: block b
// sits at word 16 + b W of the stream.
#include "codec_common.cuh"

namespace ckfwi {
namespace {

constexpr uint32_t RATE_VERSION = 2u;
constexpr int RATE_EMIN = -100;
constexpr int RWARPS = 4;              // warps (blocks) per CTA

__constant__ Perm c_rperm3 = make_perm(3);
__constant__ Perm c_rperm2 = make_perm(2);
template <int DIMS> __device__ __forceinline__ int rperm(int r) { return DIMS == 3 ? c_rperm3.p[r] : c_rperm2.p[r]; }

__host__ __device__ inline long long rate_block_words(int dims, int rate) { return ((long long)rate * (dims == 3 ? 64 : 16) + 31) / 32; }

// value index i of a block -> its clamped offset in the field
template <int DIMS>
__device__ __forceinline__ long long value_offset(const CodecView& v, const BlockPos& bp, int i, bool& inside)
{
    const int lz = DIMS == 3 ? i / 16 : i / 4;
    const int ly = DIMS == 3 ? (i / 4) % 4 : 0;
    const int lx = i % 4;
    const int z = 4 * bp.bz + lz, y = DIMS == 3 ? 4 * bp.by + ly : 0, x = 4 * bp.bx + lx;
    inside = z < v.nz && y < v.ny && x < v.nx;
    return (long long)min(z, v.nz - 1) * v.pz + (long long)min(y, v.ny - 1) * v.py + min(x, v.nx - 1);
}

// lifting of the warp's block in shared memory s[V] (x rows, then y, then z)
template <int DIMS>
__device__ __forceinline__ void warp_xform_fwd(int32_t* s, int lane)
{
    if (DIMS == 3) {
        if (lane < 16) lift_fwd(s[4 * lane], s[4 * lane + 1], s[4 * lane + 2], s[4 * lane + 3]);
        __syncwarp();
        if (lane < 16) {
            const int b = 16 * (lane / 4) + lane % 4;
            lift_fwd(s[b], s[b + 4], s[b + 8], s[b + 12]);
        }
        __syncwarp();
        if (lane < 16) lift_fwd(s[lane], s[lane + 16], s[lane + 32], s[lane + 48]);
    } else {
        if (lane < 4) lift_fwd(s[4 * lane], s[4 * lane + 1], s[4 * lane + 2], s[4 * lane + 3]);
        __syncwarp();
        if (lane < 4) lift_fwd(s[lane], s[lane + 4], s[lane + 8], s[lane + 12]);
    }
    __syncwarp();
}

template <int DIMS>
__device__ __forceinline__ void warp_xform_inv(int32_t* s, int lane)
{
    if (DIMS == 3) {
        if (lane < 16) lift_inv(s[lane], s[lane + 16], s[lane + 32], s[lane + 48]);
        __syncwarp();
        if (lane < 16) {
            const int b = 16 * (lane / 4) + lane % 4;
            lift_inv(s[b], s[b + 4], s[b + 8], s[b + 12]);
        }
        __syncwarp();
        if (lane < 16) lift_inv(s[4 * lane], s[4 * lane + 1], s[4 * lane + 2], s[4 * lane + 3]);
    } else {
        if (lane < 4) lift_inv(s[lane], s[lane + 4], s[lane + 8], s[lane + 12]);
        __syncwarp();
        if (lane < 4) lift_inv(s[4 * lane], s[4 * lane + 1], s[4 * lane + 2], s[4 * lane + 3]);
    }
    __syncwarp();
}

// Bit writer with a budget: appends the low n bits of v while they fit;
// `full` once a bit was dropped.  Completed words go to the warp's buffer
// (lane 0 stores; every lane keeps the same state).
struct RateW {
    uint32_t* w;
    unsigned long long acc;
    int nacc, nw, left;
    bool full;
    __device__ __forceinline__ void put(unsigned long long v, int n, int lane)   // n <= 64
    {
        if (full || n <= 0) return;
        if (n > left) {
            n = left;
            full = true;
        }
        left -= n;
        while (n > 0) {
            const int k = min(n, 32);
            const unsigned long long part = k == 64 ? v : (v & ((1ull << k) - 1ull));
            acc |= part << nacc;
            nacc += k;
            v = k == 64 ? 0 : (v >> k);
            n -= k;
            if (nacc >= 32) {
                if (lane == 0) w[nw] = (uint32_t)acc;
                ++nw;
                acc >>= 32;
                nacc -= 32;
            }
        }
    }
    __device__ __forceinline__ void flush(int lane)
    {
        if (nacc > 0) {
            if (lane == 0) w[nw] = (uint32_t)acc;
            ++nw;
            acc = 0;
            nacc = 0;
        }
    }
};

__device__ __forceinline__ unsigned long long lowbits(int n) { return n >= 64 ? ~0ull : ((1ull << n) - 1ull); }

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
__global__ void __launch_bounds__(RWARPS * 32) rate_enc_kernel(const float* __restrict__ x, CodecView v, Geo G,
                                                               int rate, uint32_t* __restrict__ out,
                                                               const long long* base_word, long long cap_words,
                                                               int* err)
{
    constexpr int V = DIMS == 3 ? 64 : 16;
    __shared__ int32_t sv[RWARPS][64];
    __shared__ uint32_t sw[RWARPS][64];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const long long b = (long long)blockIdx.x * RWARPS + wi;
    if (b >= G.nblocks) return;
    const long long W = rate_block_words(DIMS, rate);
    const long long base = *base_word;
    if (base + HDR + G.nblocks * W > cap_words) return;     // the header kernel raised the error
    uint32_t* o = out + base + HDR + b * W;
    int32_t* s = sv[wi];
    uint32_t* bw = sw[wi];
    const BlockPos bp = block_pos(G, b);

    // values l and l + 32 (2D: lanes 0..15 hold one each)
    bool in0, in1;
    const bool has0 = lane < V, has1 = lane + 32 < V;
    const float f0 = has0 ? __ldg(x + value_offset<DIMS>(v, bp, lane, in0)) : 0.0f;
    const float f1 = has1 ? __ldg(x + value_offset<DIMS>(v, bp, lane + 32, in1)) : 0.0f;
    const uint32_t u0 = __float_as_uint(f0), u1 = __float_as_uint(f1);
    const bool bad = __any_sync(0xffffffffu, (has0 && !isfinite(f0)) || (has1 && !isfinite(f1)));
    const bool nz0 = (u0 & 0x7FFFFFFFu) != 0, nz1 = (u1 & 0x7FFFFFFFu) != 0;
    auto expo = [](uint32_t u) { const int be = (int)((u >> 23) & 0xFF); return (be > 0 ? be : 1) - 127; };
    const int e0 = nz0 ? expo(u0) : -1000, e1 = nz1 ? expo(u1) : -1000;
    const int emax = __reduce_max_sync(0xffffffffu, max(e0, e1));
    for (int k = lane; k < W; k += 32) bw[k] = 0u;
    __syncwarp();
    if (bad || emax < RATE_EMIN) {        // zero-coded block (no non-zero value: emax = -1000)
        if (bad && lane == 0) atomicOr(err, 1);
        if (bad && lane == 0) atomicOr(out + base + 9, 1u);
        for (int k = lane; k < W; k += 32) o[k] = 0u;
        return;
    }
    auto to_int = [&](uint32_t u, bool nzv) {
        const int be = (int)((u >> 23) & 0xFF);
        const uint32_t M = (u & 0x7FFFFFu) | (be > 0 ? 0x800000u : 0u);
        const int sh = emax - ((be > 0 ? be : 1) - 127);
        uint32_t mag = sh >= 32 ? 0u : (M >> sh);
        if (!nzv) mag = 0;
        return (u >> 31) ? -(int32_t)mag : (int32_t)mag;
    };
    if (has0) s[lane] = to_int(u0, nz0);
    if (has1) s[lane + 32] = to_int(u1, nz1);
    __syncwarp();
    warp_xform_fwd<DIMS>(s, lane);
    const uint32_t n0 = has0 ? nega(s[rperm<DIMS>(lane)]) : 0u;
    const uint32_t n1 = has1 ? nega(s[rperm<DIMS>(lane + 32)]) : 0u;
    const uint32_t orall = __reduce_or_sync(0xffffffffu, n0 | n1);
    const int ptop = orall ? 31 - __clz(orall) : 0;

    RateW wr{bw, 0ull, 0, 0, (int)(W * 32), false};
    wr.put(1u, 1, lane);
    wr.put((unsigned long long)(emax + 127), 8, lane);
    wr.put((unsigned long long)ptop, 5, lane);
    int sgn = 0;   // s: coefficients already significant
    for (int p = ptop; p >= 0 && !wr.full; --p) {
        const unsigned long long lo = __ballot_sync(0xffffffffu, (n0 >> p) & 1u);
        const unsigned long long hi = __ballot_sync(0xffffffffu, (n1 >> p) & 1u);
        const unsigned long long m = lo | (hi << 32);
        wr.put(m & lowbits(sgn), sgn, lane);
        while (!wr.full && sgn < V) {
            const unsigned long long rest = m >> sgn;
            wr.put(rest ? 1u : 0u, 1, lane);
            if (!rest || wr.full) break;
            const int f = __ffsll((long long)rest) - 1;   // zeros before the next significant one
            wr.put(1ull << f, f + 1, lane);
            sgn += f + 1;
        }
    }
    wr.flush(lane);
    __syncwarp();
    for (int k = lane; k < W; k += 32) o[k] = bw[k];
}

// Bit reader over a block held in shared memory, with the same budget.
struct RateR {
    const uint32_t* w;
    int pos, end;
    bool more;
    __device__ __forceinline__ unsigned long long peek64() const   // 64 bits from pos, zeros past the end
    {
        unsigned long long r = 0;
        const int k = pos >> 5, sh = pos & 31;
        const int nwd = end >> 5;
        const unsigned long long a = k < nwd ? w[k] : 0u, b = k + 1 < nwd ? w[k + 1] : 0u,
                                 c = k + 2 < nwd ? w[k + 2] : 0u;
        r = (a | (b << 32)) >> sh;
        if (sh) r |= c << (64 - sh);
        return r;
    }
    // n <= 64 bits; stops (more = false) when the budget runs out
    __device__ __forceinline__ unsigned long long get(int n)
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
__global__ void __launch_bounds__(RWARPS * 32) rate_dec_kernel(const uint32_t* __restrict__ in, const long long* base_word,
                                                               long long cap_words, Geo G, int rate, CodecView v,
                                                               float* __restrict__ x, int* err)
{
    constexpr int V = DIMS == 3 ? 64 : 16;
    __shared__ int32_t sv[RWARPS][64];
    __shared__ uint32_t sw[RWARPS][66];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const long long b = (long long)blockIdx.x * RWARPS + wi;
    if (b >= G.nblocks) return;
    const long long W = rate_block_words(DIMS, rate);
    const long long base = *base_word;
    if (base < 0 || base + HDR + G.nblocks * W > cap_words) {
        if (lane == 0) atomicOr(err, 4);
        return;
    }
    const uint32_t* h = in + base;
    if (h[0] != MAGIC || h[1] != ((uint32_t)DIMS | (RATE_VERSION << 8)) || h[2] != (uint32_t)G.nz ||
        h[3] != (uint32_t)G.ny || h[4] != (uint32_t)G.nx || h[5] != (uint32_t)G.nblocks ||
        h[7] != (uint32_t)(G.nblocks * W) || h[8] != (uint32_t)rate) {
        if (lane == 0) atomicOr(err, 4);
        return;
    }
    const uint32_t* blk = h + HDR + b * W;
    uint32_t* bw = sw[wi];
    int32_t* s = sv[wi];
    for (int k = lane; k < W; k += 32) bw[k] = __ldg(blk + k);
    __syncwarp();
    RateR rd{bw, 0, (int)(W * 32), true};
    uint32_t n0 = 0, n1 = 0;
    int emax = 0;
    const bool coded = rd.get(1) != 0;
    if (coded) {
        emax = (int)rd.get(8) - 127;
        const int ptop = (int)rd.get(5);
        int sgn = 0;
        for (int p = ptop; p >= 0 && rd.more; --p) {
            // verbatim bits of the significant coefficients (as many as the budget holds)
            const int k = min(sgn, rd.end - rd.pos);
            unsigned long long m = rd.get(k);
            if (k < sgn) rd.more = false;
            while (rd.more && sgn < V) {
                const unsigned long long g = rd.get(1);
                if (!rd.more || !g) break;
                // bits of coefficients sgn, sgn+1, ... up to and including the first set one
                const int avail = min(V - sgn, rd.end - rd.pos);
                const unsigned long long win = rd.peek64() & lowbits(avail);
                if (win) {
                    const int f = __ffsll((long long)win) - 1;
                    m |= 1ull << (sgn + f);
                    rd.pos += f + 1;
                    sgn += f + 1;
                } else {
                    rd.pos += avail;
                    sgn += avail;
                    if (sgn < V) rd.more = false;   // the budget ended inside the run
                }
            }
            n0 |= (uint32_t)((m >> lane) & 1ull) << p;
            n1 |= (uint32_t)((m >> (lane + 32)) & 1ull) << p;
        }
    }
    const bool has0 = lane < V, has1 = lane + 32 < V;
    float f0 = 0.0f, f1 = 0.0f;
    if (coded) {
        if (has0) s[rperm<DIMS>(lane)] = unnega(n0);
        if (has1) s[rperm<DIMS>(lane + 32)] = unnega(n1);
        __syncwarp();
        warp_xform_inv<DIMS>(s, lane);
        const float sc = pow2f(max(emax - 23, -126));
        if (has0) f0 = __fmul_rn(__int2float_rn(s[lane]), sc);
        if (has1) f1 = __fmul_rn(__int2float_rn(s[lane + 32]), sc);
    }
    const BlockPos bp = block_pos(G, b);
    bool in0 = false, in1 = false;
    if (has0) {
        const long long o = value_offset<DIMS>(v, bp, lane, in0);
        if (in0) x[o] = f0;
    }
    if (has1) {
        const long long o = value_offset<DIMS>(v, bp, lane + 32, in1);
        if (in1) x[o] = f1;
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
    const unsigned nb = (unsigned)((G.nblocks + RWARPS - 1) / RWARPS);
    rate_header_kernel<<<1, 32, 0, s>>>(out, base_word, cap_words, next_word, G, rate, err, stat_words);
    if (v.dims == 3) rate_enc_kernel<3><<<nb, RWARPS * 32, 0, s>>>(x, v, G, rate, out, base_word, cap_words, err);
    else rate_enc_kernel<2><<<nb, RWARPS * 32, 0, s>>>(x, v, G, rate, out, base_word, cap_words, err);
    return cudaGetLastError();
}

cudaError_t codec_rate_decompress_dev(const uint32_t* in, const long long* base_word, long long cap_words,
                                      const CodecView& v, int rate, float* x, int* err, cudaStream_t s)
{
    if (rate < 1 || rate > 32) return cudaErrorInvalidValue;
    const Geo G = make_geo(v.dims, v.nz, v.ny, v.nx);
    const unsigned nb = (unsigned)((G.nblocks + RWARPS - 1) / RWARPS);
    if (v.dims == 3) rate_dec_kernel<3><<<nb, RWARPS * 32, 0, s>>>(in, base_word, cap_words, G, rate, v, x, err);
    else rate_dec_kernel<2><<<nb, RWARPS * 32, 0, s>>>(in, base_word, cap_words, G, rate, v, x, err);
    return cudaGetLastError();
}

}  // namespace ckfwi
