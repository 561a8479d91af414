/*
 * Plain C oracle of the fixed-accuracy block-transform codec used for
 * compressed checkpoints.  TEST INFRASTRUCTURE ONLY (see fwi_oracle.c).
 *
 * The paper compresses checkpoints with ZFP in fixed-tolerance mode, an
 * absolute point-wise error bound (Sec. 2.2 "Lossy Compression").  This is
 * not ZFP and is not bit-compatible with it; it is a codec of the same
 * family (block floating point, decorrelating lifting transform, ordering by
 * sequency, negabinary, embedded bit-plane coding with group tests) whose
 * every step is specified below and implemented independently here and in
 * the CUDA library.  Identical float input gives identical streams.
 *
 * Field: float32, logical shape (nz, ny, nx), x fastest; 2D fields have
 * ny = 1 and use 4x4 blocks over (z, x).  tol > 0 is an absolute bound;
 * tol_f = the largest float <= tol; tol must be >= 2^-90.
 *
 * Blocks: 4^d cubes, block id b = (bz*nby + by)*nbx + bx; partial blocks
 * read the nearest valid sample (index clamped to the last one per axis).
 * Values in a block: V = 64 (3D) or 16 (2D), local index (lz*4+ly)*4+lx.
 *
 * Per block:
 *  1. zero block if max |x| <= tol_f: one bit 0.  Non-finite input sets the
 *     NONFINITE flag and is coded as a zero block.
 *  2. Emax = max over non-zero x of (max(biased exponent,1) - 127).
 *  3. i = trunc(x * 2^(23-Emax)) computed on the bits: significand M
 *     (with hidden bit for normal numbers) shifted right by Emax - Eeff;
 *     |i| < 2^24, exact, error < 2^(Emax-23).
 *  4. lifting transform of every 4-vector along x, then y (3D), then z,
 *     in 32-bit two's-complement wrap-around arithmetic, ">>" arithmetic:
 *        d3 = x3 - 2 x2 + x1      (linear extrapolation residual)
 *        d1 = x1 - ((x0 + x2) >> 1)   (linear interpolation residual)
 *        D  = x2 - x0,  S = x0 + (D >> 1)
 *     output order (S, D, d1, d3).  The inverse is exact:
 *        x0 = S - (D >> 1), x2 = D + x0, x1 = d1 + ((x0 + x2) >> 1),
 *        x3 = d3 + 2 x2 - x1.
 *     Growth is at most 4x per axis, so coefficients stay below 2^30.
 *  5. coefficients ordered by (kz+ky+kx, kz, ky, kx) ascending (2D:
 *     (kz+kx, kz, kx)), then mapped to negabinary
 *        n = (c + 0xAAAAAAAA) ^ 0xAAAAAAAA   (mod 2^32).
 *  6. ptop = index of the highest set bit over all n.
 *     T = floor(tol_f * 2^(23-Emax)).  A candidate lowest plane pbot keeps
 *     bits pbot..31 of every n; it is accepted when the exact inverse of
 *     steps 5 and 4 reproduces every i within T - 2 (this covers the
 *     truncation of step 3 and the rounding of the decoder's int->float
 *     conversion, so |x - x_hat| <= tol holds on every value).  The search
 *     starts at min(ptop, max(0, floor(log2 T) - 1)) and goes down; if
 *     T < 2 or Emax >= 126 (values near the float range limit) the block is
 *     stored raw.
 *  7. stream: 1, 0, Emax+127 (8 bits), ptop (5), pbot (5), then planes
 *     ptop..pbot, each coded against the count s of coefficients already
 *     significant (s = 0 at the first plane):
 *        the plane bits of coefficients 0..s-1 verbatim, then repeatedly a
 *        group-test bit "is any of coefficients s..V-1 set in this plane";
 *        after a 1, the bits of coefficients s, s+1, ... up to and
 *        including the first set one, s moving past it.
 *     raw block: 1, 1, then the V float bit patterns (32 bits each).
 *     A coded block whose stream would be longer than its raw form
 *     (2 + 32 V bits) is stored raw, so no block exceeds 2 + 32 V bits.
 *     Bits are written LSB first into 32-bit words.
 *  Decoding: planes below pbot are zero; inverse negabinary, order and
 *  lifting; x_hat = float(i_hat) * 2^(Emax-23).
 *
 * Container (32-bit words):
 *   [0] magic 0x31435442  [1] dims | version<<8  [2..4] nz, ny, nx
 *   [5] nblocks  [6] nchunks  [7] payload words  [8] tol_f bits
 *   [9] flags (bit0 NONFINITE)  [10..15] 0
 *   chunk table: nchunks words, payload word offset of each chunk
 *   size table: nblocks uint16 (bits of each block), 2 per word, even
 *               block in the low half
 *   payload: chunks of 32 consecutive blocks, each chunk starting on a
 *            word boundary, blocks back to back inside it; unused bits 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CODEC_MAGIC 0x31435442u
#define CODEC_VERSION 1u
#ifndef CODEC_GUARD
#define CODEC_GUARD 1
#endif
#define CODEC_HDR_WORDS 16
#define CHUNK_BLOCKS 32
#define CODEC_RATE_VERSION 2u   /* fixed-rate streams (see "fixed-rate mode" below) */

enum { C_OK = 0, C_EINVAL = -1, C_ENOMEM = -2, C_OVERFLOW = -3, C_CORRUPT = -4 };

/* ---------- geometry ---------- */
typedef struct {
    int dims, nz, ny, nx;
    int nbz, nby, nbx, V;
    long nblocks, nchunks;
} cgeom;

static int geom_init(cgeom* G, int dims, int nz, int ny, int nx)
{
    if ((dims != 2 && dims != 3) || nz < 1 || nx < 1 || ny < 1) return C_EINVAL;
    if (dims == 2 && ny != 1) return C_EINVAL;
    G->dims = dims; G->nz = nz; G->ny = ny; G->nx = nx;
    G->nbz = (nz + 3) / 4;
    G->nby = (dims == 3) ? (ny + 3) / 4 : 1;
    G->nbx = (nx + 3) / 4;
    G->V = (dims == 3) ? 64 : 16;
    G->nblocks = (long)G->nbz * G->nby * G->nbx;
    G->nchunks = (G->nblocks + CHUNK_BLOCKS - 1) / CHUNK_BLOCKS;
    return C_OK;
}

static int max_block_bits(const cgeom* G) { return 2 + 32 * G->V; }

static int decompress_rate(const cgeom* G, const uint32_t* in, size_t nwords, float* x);

static long table_words(const cgeom* G) { return CODEC_HDR_WORDS + G->nchunks + (G->nblocks + 1) / 2; }

long long codec_bound_words(int dims, int nz, int ny, int nx)
{
    cgeom G;
    if (geom_init(&G, dims, nz, ny, nx) != C_OK) return C_EINVAL;
    long per_chunk = (CHUNK_BLOCKS * (long)max_block_bits(&G) + 31) / 32;
    return table_words(&G) + G.nchunks * per_chunk;
}

/* ---------- bit I/O ---------- */
typedef struct { uint32_t* w; long cap_bits; long pos; int overflow; } bitw;

static void put_bit(bitw* B, uint32_t bit)
{
    if (B->pos >= B->cap_bits) { B->overflow = 1; return; }
    if (bit & 1u) B->w[B->pos >> 5] |= 1u << (B->pos & 31);
    B->pos++;
}

static void put_bits(bitw* B, uint32_t v, int n)
{
    for (int k = 0; k < n; ++k) put_bit(B, (v >> k) & 1u);
}

typedef struct { const uint32_t* w; long end; long pos; int bad; } bitr;

static uint32_t get_bit(bitr* B)
{
    if (B->pos >= B->end) { B->bad = 1; return 0; }
    uint32_t b = (B->w[B->pos >> 5] >> (B->pos & 31)) & 1u;
    B->pos++;
    return b;
}

static uint32_t get_bits(bitr* B, int n)
{
    uint32_t v = 0;
    for (int k = 0; k < n; ++k) v |= get_bit(B) << k;
    return v;
}

/* ---------- arithmetic helpers (two's complement wrap-around) ---------- */
static int32_t wadd(int32_t a, int32_t b) { return (int32_t)((uint32_t)a + (uint32_t)b); }
static int32_t wsub(int32_t a, int32_t b) { return (int32_t)((uint32_t)a - (uint32_t)b); }
static int32_t half(int32_t a) { return a >> 1; }   /* arithmetic shift: floor(a/2) */

static void fwd_lift(int32_t* v, int stride)
{
    int32_t x0 = v[0], x1 = v[stride], x2 = v[2 * stride], x3 = v[3 * stride];
    int32_t d3 = wadd(wsub(x3, wadd(x2, x2)), x1);
    int32_t d1 = wsub(x1, half(wadd(x0, x2)));
    int32_t D = wsub(x2, x0);
    int32_t S = wadd(x0, half(D));
    v[0] = S; v[stride] = D; v[2 * stride] = d1; v[3 * stride] = d3;
}

static void inv_lift(int32_t* v, int stride)
{
    int32_t S = v[0], D = v[stride], d1 = v[2 * stride], d3 = v[3 * stride];
    int32_t x0 = wsub(S, half(D));
    int32_t x2 = wadd(D, x0);
    int32_t x1 = wadd(d1, half(wadd(x0, x2)));
    int32_t x3 = wsub(wadd(d3, wadd(x2, x2)), x1);
    v[0] = x0; v[stride] = x1; v[2 * stride] = x2; v[3 * stride] = x3;
}

/* Block transform: x rows, then y (3D), then z; block stored (lz,ly,lx). */
static void fwd_xform(int32_t* b, int dims)
{
    if (dims == 3) {
        for (int z = 0; z < 4; ++z) for (int y = 0; y < 4; ++y) fwd_lift(b + 16 * z + 4 * y, 1);
        for (int z = 0; z < 4; ++z) for (int x = 0; x < 4; ++x) fwd_lift(b + 16 * z + x, 4);
        for (int y = 0; y < 4; ++y) for (int x = 0; x < 4; ++x) fwd_lift(b + 4 * y + x, 16);
    } else {
        for (int z = 0; z < 4; ++z) fwd_lift(b + 4 * z, 1);
        for (int x = 0; x < 4; ++x) fwd_lift(b + x, 4);
    }
}

static void inv_xform(int32_t* b, int dims)
{
    if (dims == 3) {
        for (int y = 0; y < 4; ++y) for (int x = 0; x < 4; ++x) inv_lift(b + 4 * y + x, 16);
        for (int z = 0; z < 4; ++z) for (int x = 0; x < 4; ++x) inv_lift(b + 16 * z + x, 4);
        for (int z = 0; z < 4; ++z) for (int y = 0; y < 4; ++y) inv_lift(b + 16 * z + 4 * y, 1);
    } else {
        for (int x = 0; x < 4; ++x) inv_lift(b + x, 4);
        for (int z = 0; z < 4; ++z) inv_lift(b + 4 * z, 1);
    }
}

/* perm[r] = local index of the r-th coefficient in sequency order. */
static void sequency_order(int dims, int* perm)
{
    int V = (dims == 3) ? 64 : 16;
    int key[64];
    for (int i = 0; i < V; ++i) {
        int kz, ky, kx;
        if (dims == 3) { kz = i / 16; ky = (i / 4) % 4; kx = i % 4; }
        else { kz = i / 4; ky = 0; kx = i % 4; }
        key[i] = (kz + ky + kx) * 4096 + kz * 256 + ky * 16 + kx;
        perm[i] = i;
    }
    /* insertion sort by key */
    for (int a = 1; a < V; ++a) {
        int p = perm[a], j = a - 1;
        while (j >= 0 && key[perm[j]] > key[p]) { perm[j + 1] = perm[j]; --j; }
        perm[j + 1] = p;
    }
}

static uint32_t to_nega(int32_t c) { return ((uint32_t)c + 0xAAAAAAAAu) ^ 0xAAAAAAAAu; }
static int32_t from_nega(uint32_t n) { return (int32_t)((n ^ 0xAAAAAAAAu) - 0xAAAAAAAAu); }

static float f_of_bits(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint32_t bits_of_f(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* largest float <= t (t > 0) */
static float tol_to_float(double t)
{
    float f = (float)t;
    if ((double)f > t) f = nextafterf(f, 0.0f);
    return f;
}

/* 2^e as a float, -126 <= e <= 127 */
static float pow2f(int e) { return f_of_bits((uint32_t)(e + 127) << 23); }

static void gather_block(const cgeom* G, const float* x, long b, float* v)
{
    long bx = b % G->nbx, t = b / G->nbx;
    long by = t % G->nby, bz = t / G->nby;
    for (int i = 0; i < G->V; ++i) {
        int lz, ly, lx;
        if (G->dims == 3) { lz = i / 16; ly = (i / 4) % 4; lx = i % 4; }
        else { lz = i / 4; ly = 0; lx = i % 4; }
        long z = 4 * bz + lz, y = (G->dims == 3) ? 4 * by + ly : 0, xx = 4 * bx + lx;
        if (z > G->nz - 1) z = G->nz - 1;
        if (y > G->ny - 1) y = G->ny - 1;
        if (xx > G->nx - 1) xx = G->nx - 1;
        v[i] = x[(z * G->ny + y) * G->nx + xx];
    }
}

/* Encode one block; returns its bit count (bits appended to B). */
static int encode_block(const cgeom* G, const int* perm, const float* v, float tol_f,
                        bitw* B, int* nonfinite)
{
    const int V = G->V;
    const long start = B->pos;
    float amax = 0.0f;
    int bad = 0;
    for (int i = 0; i < V; ++i) {
        if (!isfinite(v[i])) bad = 1;
        float a = fabsf(v[i]);
        if (a > amax) amax = a;
    }
    if (bad) { *nonfinite = 1; put_bit(B, 0); return (int)(B->pos - start); }
    if (amax <= tol_f) { put_bit(B, 0); return (int)(B->pos - start); }

    int emax = -1000;
    for (int i = 0; i < V; ++i) {
        uint32_t u = bits_of_f(v[i]);
        if ((u & 0x7FFFFFFFu) == 0) continue;
        int be = (int)((u >> 23) & 0xFF);
        int e = (be > 0 ? be : 1) - 127;
        if (e > emax) emax = e;
    }
    int32_t iv[64], cf[64], tr[64];
    for (int i = 0; i < V; ++i) {
        uint32_t u = bits_of_f(v[i]);
        int be = (int)((u >> 23) & 0xFF);
        uint32_t M = (u & 0x7FFFFFu) | (be > 0 ? 0x800000u : 0u);
        int e = (be > 0 ? be : 1) - 127;
        int sh = emax - e;
        uint32_t mag = (sh >= 32) ? 0u : (M >> sh);
        if ((u & 0x7FFFFFFFu) == 0) mag = 0;
        iv[i] = (u >> 31) ? -(int32_t)mag : (int32_t)mag;
    }
    for (int i = 0; i < V; ++i) cf[i] = iv[i];
    fwd_xform(cf, G->dims);
    uint32_t nb[64], orall = 0;
    for (int r = 0; r < V; ++r) { nb[r] = to_nega(cf[perm[r]]); orall |= nb[r]; }
    int ptop = 31;
    while (ptop > 0 && !((orall >> ptop) & 1u)) --ptop;

    float Tf = tol_f * pow2f(23 - emax);
    long T = (long)Tf;                         /* floor for positive values */
    int pbot = -1;
    if (T >= 2 && emax < 126) {
        int lg = 0;
        while (lg < 62 && (T >> (lg + 1)) != 0) ++lg;   /* floor(log2 T) */
        int p0 = lg - CODEC_GUARD;
        if (p0 < 0) p0 = 0;
        if (p0 > ptop) p0 = ptop;
        for (int p = p0; p >= 0; --p) {
            uint32_t mask = (p >= 32) ? 0u : ~((1u << p) - 1u);
            for (int r = 0; r < V; ++r) tr[perm[r]] = from_nega(nb[r] & mask);
            inv_xform(tr, G->dims);
            int ok = 1;
            for (int i = 0; i < V && ok; ++i) {
                long diff = (long)iv[i] - (long)tr[i];
                if (diff < 0) diff = -diff;
                if (diff > T - 2) ok = 0;
            }
            if (ok) { pbot = p; break; }
        }
    }
    const int raw_bits = 2 + 32 * V;
    if (pbot >= 0) {
        /* the coded stream, built aside and kept if not longer than raw */
        uint32_t tmp[160];
        memset(tmp, 0, sizeof(tmp));
        bitw C = {tmp, 160 * 32, 0, 0};
        put_bit(&C, 1);
        put_bit(&C, 0);
        put_bits(&C, (uint32_t)(emax + 127), 8);
        put_bits(&C, (uint32_t)ptop, 5);
        put_bits(&C, (uint32_t)pbot, 5);
        int s = 0;
        for (int p = ptop; p >= pbot; --p) {
            uint32_t plane[64];
            for (int r = 0; r < V; ++r) plane[r] = (nb[r] >> p) & 1u;
            for (int r = 0; r < s; ++r) put_bit(&C, plane[r]);
            while (s < V) {
                uint32_t any = 0;
                for (int r = s; r < V; ++r) any |= plane[r];
                put_bit(&C, any);
                if (!any) break;
                for (;;) {
                    uint32_t bit = plane[s];
                    put_bit(&C, bit);
                    ++s;
                    if (bit) break;
                }
            }
        }
        if (C.pos <= raw_bits) {
            for (long k = 0; k < C.pos; ++k) put_bit(B, (tmp[k >> 5] >> (k & 31)) & 1u);
            return (int)(B->pos - start);
        }
    }
    put_bit(B, 1);                              /* raw block */
    put_bit(B, 1);
    for (int i = 0; i < V; ++i) put_bits(B, bits_of_f(v[i]), 32);
    return (int)(B->pos - start);
}

/* Decode one block from B into v (V values); returns 0 or C_CORRUPT. */
static int decode_block(const cgeom* G, const int* perm, bitr* B, float* v)
{
    const int V = G->V;
    if (!get_bit(B)) {
        for (int i = 0; i < V; ++i) v[i] = 0.0f;
        return B->bad ? C_CORRUPT : C_OK;
    }
    if (get_bit(B)) {
        for (int i = 0; i < V; ++i) v[i] = f_of_bits(get_bits(B, 32));
        return B->bad ? C_CORRUPT : C_OK;
    }
    int emax = (int)get_bits(B, 8) - 127;
    int ptop = (int)get_bits(B, 5);
    int pbot = (int)get_bits(B, 5);
    if (emax < -126 || emax > 127 || pbot > ptop) return C_CORRUPT;
    uint32_t nb[64];
    for (int r = 0; r < V; ++r) nb[r] = 0;
    int s = 0;
    for (int p = ptop; p >= pbot; --p) {
        for (int r = 0; r < s; ++r) nb[r] |= get_bit(B) << p;
        while (s < V) {
            if (!get_bit(B)) break;
            for (;;) {
                if (s >= V) return C_CORRUPT;
                uint32_t bit = get_bit(B);
                nb[s] |= bit << p;
                ++s;
                if (bit) break;
            }
        }
        if (B->bad) return C_CORRUPT;
    }
    int32_t tr[64];
    for (int r = 0; r < V; ++r) tr[perm[r]] = from_nega(nb[r]);
    inv_xform(tr, G->dims);
    float sc = pow2f(emax - 23 < -126 ? -126 : emax - 23);
    /* emax >= -91 for any stream the encoder writes (tol >= 2^-90), so the
     * clamp above never applies to valid input. */
    for (int i = 0; i < V; ++i) v[i] = (float)tr[i] * sc;
    return B->bad ? C_CORRUPT : C_OK;
}

static void scatter_block(const cgeom* G, float* x, long b, const float* v)
{
    long bx = b % G->nbx, t = b / G->nbx;
    long by = t % G->nby, bz = t / G->nby;
    for (int i = 0; i < G->V; ++i) {
        int lz, ly, lx;
        if (G->dims == 3) { lz = i / 16; ly = (i / 4) % 4; lx = i % 4; }
        else { lz = i / 4; ly = 0; lx = i % 4; }
        long z = 4 * bz + lz, y = (G->dims == 3) ? 4 * by + ly : 0, xx = 4 * bx + lx;
        if (z >= G->nz || y >= G->ny || xx >= G->nx) continue;
        x[(z * G->ny + y) * G->nx + xx] = v[i];
    }
}

/* Compress x into out (cap words).  Returns the words used, or < 0.
 * *flags receives bit0 = NONFINITE. */
long long codec_compress(int dims, int nz, int ny, int nx, const float* x, double tol,
                         uint32_t* out, size_t cap, int* flags)
{
    cgeom G;
    if (geom_init(&G, dims, nz, ny, nx) != C_OK || !x || !out) return C_EINVAL;
    if (!(tol >= ldexp(1.0, -90)) || !isfinite(tol)) return C_EINVAL;
    const long tw = table_words(&G);
    if ((long)cap < tw) return C_OVERFLOW;
    memset(out, 0, sizeof(uint32_t) * cap);
    const float tol_f = tol_to_float(tol);
    int perm[64];
    sequency_order(dims, perm);
    uint32_t* chunk_off = out + CODEC_HDR_WORDS;
    uint16_t* sizes = (uint16_t*)malloc(sizeof(uint16_t) * (G.nblocks + 1));
    if (!sizes) return C_ENOMEM;
    uint32_t* payload = out + tw;
    long cap_bits = ((long)cap - tw) * 32;
    int nonfinite = 0;
    long chunk_word = 0;
    float v[64];
    for (long c = 0; c < G.nchunks; ++c) {
        chunk_off[c] = (uint32_t)chunk_word;
        bitw B = {payload + chunk_word, cap_bits - chunk_word * 32, 0, 0};
        long b0 = c * CHUNK_BLOCKS;
        long b1 = b0 + CHUNK_BLOCKS < G.nblocks ? b0 + CHUNK_BLOCKS : G.nblocks;
        for (long b = b0; b < b1; ++b) {
            gather_block(&G, x, b, v);
            int nbits = encode_block(&G, perm, v, tol_f, &B, &nonfinite);
            sizes[b] = (uint16_t)nbits;
        }
        if (B.overflow) { free(sizes); return C_OVERFLOW; }
        chunk_word += (B.pos + 31) / 32;
    }
    uint32_t* st = out + CODEC_HDR_WORDS + G.nchunks;
    for (long b = 0; b < G.nblocks; ++b) {
        if (b & 1) st[b >> 1] |= (uint32_t)sizes[b] << 16;
        else st[b >> 1] |= (uint32_t)sizes[b];
    }
    free(sizes);
    out[0] = CODEC_MAGIC;
    out[1] = (uint32_t)dims | (CODEC_VERSION << 8);
    out[2] = (uint32_t)nz; out[3] = (uint32_t)ny; out[4] = (uint32_t)nx;
    out[5] = (uint32_t)G.nblocks; out[6] = (uint32_t)G.nchunks;
    out[7] = (uint32_t)chunk_word;
    out[8] = bits_of_f(tol_f);
    out[9] = nonfinite ? 1u : 0u;
    if (flags) *flags = nonfinite;
    return tw + chunk_word;
}

int codec_decompress(int dims, int nz, int ny, int nx, const uint32_t* in, size_t nwords,
                     float* x)
{
    cgeom G;
    if (geom_init(&G, dims, nz, ny, nx) != C_OK || !in || !x) return C_EINVAL;
    if (nwords >= CODEC_HDR_WORDS && in[0] == CODEC_MAGIC && in[1] == ((uint32_t)dims | (CODEC_RATE_VERSION << 8))) {
        if (in[2] != (uint32_t)nz || in[3] != (uint32_t)ny || in[4] != (uint32_t)nx ||
            in[5] != (uint32_t)G.nblocks)
            return C_CORRUPT;
        return decompress_rate(&G, in, nwords, x);
    }
    const long tw = table_words(&G);
    if ((long)nwords < tw) return C_CORRUPT;
    if (in[0] != CODEC_MAGIC || in[1] != ((uint32_t)dims | (CODEC_VERSION << 8)) ||
        in[2] != (uint32_t)nz || in[3] != (uint32_t)ny || in[4] != (uint32_t)nx ||
        in[5] != (uint32_t)G.nblocks || in[6] != (uint32_t)G.nchunks)
        return C_CORRUPT;
    const long pw = in[7];
    if (tw + pw > (long)nwords) return C_CORRUPT;
    int perm[64];
    sequency_order(dims, perm);
    const uint32_t* chunk_off = in + CODEC_HDR_WORDS;
    const uint32_t* st = in + CODEC_HDR_WORDS + G.nchunks;
    const uint32_t* payload = in + tw;
    float v[64];
    for (long c = 0; c < G.nchunks; ++c) {
        long pos = (long)chunk_off[c] * 32;
        long b0 = c * CHUNK_BLOCKS;
        long b1 = b0 + CHUNK_BLOCKS < G.nblocks ? b0 + CHUNK_BLOCKS : G.nblocks;
        for (long b = b0; b < b1; ++b) {
            uint32_t sz = (st[b >> 1] >> ((b & 1) ? 16 : 0)) & 0xFFFFu;
            bitr B = {payload, pos + (long)sz, pos, 0};
            if (B.end > pw * 32) return C_CORRUPT;
            int s = decode_block(&G, perm, &B, v);
            if (s != C_OK || B.pos != B.end) return C_CORRUPT;
            scatter_block(&G, x, b, v);
            pos += sz;
        }
    }
    return C_OK;
}

/* Per-block statistics for tests: bits, mode (0 zero, 1 coded, 2 raw),
 * and ptop, pbot, Emax of coded blocks.  stats: [nblocks][5]. */
int codec_block_stats(int dims, int nz, int ny, int nx, const uint32_t* in, size_t nwords,
                      int* stats)
{
    cgeom G;
    if (geom_init(&G, dims, nz, ny, nx) != C_OK || !in || !stats) return C_EINVAL;
    const long tw = table_words(&G);
    if ((long)nwords < tw || in[0] != CODEC_MAGIC) return C_CORRUPT;
    const uint32_t* chunk_off = in + CODEC_HDR_WORDS;
    const uint32_t* st = in + CODEC_HDR_WORDS + G.nchunks;
    const uint32_t* payload = in + tw;
    const long pw = in[7];
    for (long c = 0; c < G.nchunks; ++c) {
        long pos = (long)chunk_off[c] * 32;
        long b0 = c * CHUNK_BLOCKS;
        long b1 = b0 + CHUNK_BLOCKS < G.nblocks ? b0 + CHUNK_BLOCKS : G.nblocks;
        for (long b = b0; b < b1; ++b) {
            uint32_t sz = (st[b >> 1] >> ((b & 1) ? 16 : 0)) & 0xFFFFu;
            bitr B = {payload, pw * 32, pos, 0};
            int* o = stats + 5 * b;
            o[0] = (int)sz;
            o[2] = o[3] = o[4] = -1000;
            if (!get_bit(&B)) o[1] = 0;
            else if (get_bit(&B)) o[1] = 2;
            else {
                o[4] = (int)get_bits(&B, 8) - 127;
                o[1] = 1;
                o[2] = (int)get_bits(&B, 5);
                o[3] = (int)get_bits(&B, 5);
            }
            pos += sz;
        }
    }
    return C_OK;
}


/* ---------- fixed-rate mode ----------
 * Sec. 2.2 lists ZFP's fixed-rate mode beside fixed tolerance: a guaranteed
 * size and no bound on the error.  This codec's fixed-rate mode:
 *   rate R bits per value, 1 <= R <= 32.  Every block occupies exactly
 *   W = ceil(R V / 32) words, a budget of 32 W bits, so a field takes
 *   16 + nblocks W words whatever its values.
 * Per block, bits LSB first from the block's first word:
 *   0                        all values are +-0, or a value is not finite
 *                            (flag NONFINITE), or Emax < -100 (every value
 *                            below 2^-99 in magnitude is flushed to zero);
 *                            the rest of the budget is zero;
 *   1, Emax+127 (8), ptop (5), then planes ptop, ptop-1, ..., 0, each coded
 *                            exactly as step 7 of the fixed-accuracy mode
 *                            (verbatim bits of the s significant
 *                            coefficients, then group tests), until the
 *                            budget is full: the first bit that does not fit
 *                            is dropped and coding stops.
 * Steps 2-5 (Emax, integers, lifting, order, negabinary) are the
 * fixed-accuracy mode's.  The decoder reads the same bits and stops at the
 * budget; a plane cut short keeps the bits read, all later bits are zero;
 * x_hat = float(i_hat) * 2^(Emax-23).  A longer budget extends a block's
 * bits and never changes the ones a shorter budget kept (the code is
 * embedded).
 * Container: the header of the fixed-accuracy mode with version 2 and
 * [7] = nblocks W, [8] = R; blocks back to back after the header, no chunk
 * or size table.
 */
#define RATE_EMIN (-100)

static long rate_block_words(const cgeom* G, int rate) { return ((long)rate * G->V + 31) / 32; }

long long codec_rate_words(int dims, int nz, int ny, int nx, int rate)
{
    cgeom G;
    if (geom_init(&G, dims, nz, ny, nx) != C_OK || rate < 1 || rate > 32) return C_EINVAL;
    return CODEC_HDR_WORDS + G.nblocks * rate_block_words(&G, rate);
}

/* append the n low bits of v while they fit in the budget; 0 once it is full */
static int put_budget(bitw* B, long end, uint32_t v, int n)
{
    for (int k = 0; k < n; ++k) {
        if (B->pos >= end) return 0;
        put_bit(B, (v >> k) & 1u);
    }
    return 1;
}

static void encode_block_rate(const cgeom* G, const int* perm, const float* v, long budget, bitw* B,
                              int* nonfinite)
{
    const int V = G->V;
    const long end = B->pos + budget;
    int bad = 0, any = 0;
    for (int i = 0; i < V; ++i) {
        if (!isfinite(v[i])) bad = 1;
        if ((bits_of_f(v[i]) & 0x7FFFFFFFu) != 0) any = 1;
    }
    if (bad) *nonfinite = 1;
    int emax = -1000;
    for (int i = 0; i < V; ++i) {
        uint32_t u = bits_of_f(v[i]);
        if ((u & 0x7FFFFFFFu) == 0) continue;
        int be = (int)((u >> 23) & 0xFF);
        int e = (be > 0 ? be : 1) - 127;
        if (e > emax) emax = e;
    }
    if (bad || !any || emax < RATE_EMIN) { put_bit(B, 0); B->pos = end; return; }
    int32_t cf[64];
    for (int i = 0; i < V; ++i) {
        uint32_t u = bits_of_f(v[i]);
        int be = (int)((u >> 23) & 0xFF);
        uint32_t M = (u & 0x7FFFFFu) | (be > 0 ? 0x800000u : 0u);
        int e = (be > 0 ? be : 1) - 127;
        int sh = emax - e;
        uint32_t mag = (sh >= 32) ? 0u : (M >> sh);
        if ((u & 0x7FFFFFFFu) == 0) mag = 0;
        cf[i] = (u >> 31) ? -(int32_t)mag : (int32_t)mag;
    }
    fwd_xform(cf, G->dims);
    uint32_t nb[64], orall = 0;
    for (int r = 0; r < V; ++r) { nb[r] = to_nega(cf[perm[r]]); orall |= nb[r]; }
    int ptop = 31;
    while (ptop > 0 && !((orall >> ptop) & 1u)) --ptop;
    int ok = put_budget(B, end, 1, 1) && put_budget(B, end, (uint32_t)(emax + 127), 8) &&
             put_budget(B, end, (uint32_t)ptop, 5);
    int s = 0;
    for (int p = ptop; p >= 0 && ok; --p) {
        uint32_t plane[64];
        for (int r = 0; r < V; ++r) plane[r] = (nb[r] >> p) & 1u;
        for (int r = 0; r < s && ok; ++r) ok = put_budget(B, end, plane[r], 1);
        while (ok && s < V) {
            uint32_t a = 0;
            for (int r = s; r < V; ++r) a |= plane[r];
            ok = put_budget(B, end, a, 1);
            if (!ok || !a) break;
            for (;;) {
                uint32_t bit = plane[s];
                ok = put_budget(B, end, bit, 1);
                if (!ok) break;
                ++s;
                if (bit) break;
            }
        }
    }
    B->pos = end;
}

/* read one bit if the budget has room; *more = 0 once it is exhausted */
static uint32_t get_budget(bitr* B, int* more)
{
    if (!*more || B->pos >= B->end) { *more = 0; return 0; }
    return get_bit(B);
}

static void decode_block_rate(const cgeom* G, const int* perm, bitr* B, float* v)
{
    const int V = G->V;
    int more = 1;
    if (!get_budget(B, &more)) {
        for (int i = 0; i < V; ++i) v[i] = 0.0f;
        return;
    }
    uint32_t e8 = 0, pt = 0;
    for (int k = 0; k < 8; ++k) e8 |= get_budget(B, &more) << k;
    for (int k = 0; k < 5; ++k) pt |= get_budget(B, &more) << k;
    const int emax = (int)e8 - 127;
    uint32_t nb[64];
    for (int r = 0; r < V; ++r) nb[r] = 0;
    int s = 0;
    for (int p = (int)pt; p >= 0 && more; --p) {
        for (int r = 0; r < s && more; ++r) nb[r] |= get_budget(B, &more) << p;
        while (more && s < V) {
            if (!get_budget(B, &more)) break;
            while (more && s < V) {
                uint32_t bit = get_budget(B, &more);
                if (!more) break;
                nb[s] |= bit << p;
                ++s;
                if (bit) break;
            }
        }
    }
    int32_t tr[64];
    for (int r = 0; r < V; ++r) tr[perm[r]] = from_nega(nb[r]);
    inv_xform(tr, G->dims);
    /* emax >= -100 for a coded block, so the scale is a normal float */
    const float sc = pow2f(emax - 23 < -126 ? -126 : emax - 23);
    for (int i = 0; i < V; ++i) v[i] = (float)tr[i] * sc;
}

/* Fixed-rate compression of x into out (cap words): returns the words used
 * (always codec_rate_words), or < 0.  *flags: bit0 NONFINITE. */
long long codec_compress_rate(int dims, int nz, int ny, int nx, const float* x, int rate, uint32_t* out,
                              size_t cap, int* flags)
{
    cgeom G;
    if (geom_init(&G, dims, nz, ny, nx) != C_OK || !x || !out || rate < 1 || rate > 32) return C_EINVAL;
    const long W = rate_block_words(&G, rate);
    const long total = CODEC_HDR_WORDS + G.nblocks * W;
    if ((long)cap < total) return C_OVERFLOW;
    memset(out, 0, sizeof(uint32_t) * total);
    int perm[64];
    sequency_order(dims, perm);
    int nonfinite = 0;
    float v[64];
    for (long b = 0; b < G.nblocks; ++b) {
        bitw B = {out + CODEC_HDR_WORDS + b * W, W * 32, 0, 0};
        gather_block(&G, x, b, v);
        encode_block_rate(&G, perm, v, W * 32, &B, &nonfinite);
    }
    out[0] = CODEC_MAGIC;
    out[1] = (uint32_t)dims | (CODEC_RATE_VERSION << 8);
    out[2] = (uint32_t)nz; out[3] = (uint32_t)ny; out[4] = (uint32_t)nx;
    out[5] = (uint32_t)G.nblocks; out[6] = 0;
    out[7] = (uint32_t)(G.nblocks * W);
    out[8] = (uint32_t)rate;
    out[9] = nonfinite ? 1u : 0u;
    if (flags) *flags = nonfinite;
    return total;
}

static int decompress_rate(const cgeom* G, const uint32_t* in, size_t nwords, float* x)
{
    const int rate = (int)in[8];
    if (rate < 1 || rate > 32 || in[6] != 0) return C_CORRUPT;
    const long W = rate_block_words(G, rate);
    if (in[7] != (uint32_t)(G->nblocks * W) || CODEC_HDR_WORDS + G->nblocks * W > (long)nwords) return C_CORRUPT;
    int perm[64];
    sequency_order(G->dims, perm);
    float v[64];
    for (long b = 0; b < G->nblocks; ++b) {
        bitr B = {in + CODEC_HDR_WORDS + b * W, W * 32, 0, 0};
        decode_block_rate(G, perm, &B, v);
        scatter_block(G, x, b, v);
    }
    return C_OK;
}

/* ---- single-step entry points used by the tests to pin the pieces ---- */
uint32_t codec_nega(int32_t c) { return to_nega(c); }
int32_t codec_from_nega(uint32_t n) { return from_nega(n); }
void codec_lift4(int32_t* v, int inverse)
{
    if (inverse) inv_lift(v, 1);
    else fwd_lift(v, 1);
}
void codec_xform(int32_t* b, int dims, int inverse)
{
    if (inverse) inv_xform(b, dims);
    else fwd_xform(b, dims);
}
void codec_order(int dims, int* perm) { sequency_order(dims, perm); }
