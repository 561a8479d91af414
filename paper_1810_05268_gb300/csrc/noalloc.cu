// Allocation-free variant of the standalone codec compression.
//
// ckfwi_codec_compress needs scratch memory (a staging slot per 32-block
// chunk for the encoded bits, the chunks' word counts and group sums, plus
// a few device scalars) and allocates it
// with cudaMalloc on first use.  Some callers cannot allow that: code that
// must not trigger cudaMalloc's implicit device synchronisation (a latency-
// critical path), processes whose device memory is entirely owned by
// another allocator or pool, and callers that have been told not to grow
// the process's device footprint after start-up.  For them,
// ckfwi_codec_compress_noalloc uses scratch that lives in this file as a
// statically sized __device__ array, so a call allocates nothing; the
// caller still passes the input field and the output buffer.
//
// The array holds the scratch of a field of NOALLOC_MAX_BLOCKS blocks (about
// 17 MB on every device that loads the library, kept until the process
// exits).
// Every call on a device shares it and it keeps the last call's contents,
// so two calls whose work overlaps on the GPU (different streams, or
// different host threads) race and corrupt each other's output; calls must
// be ordered (same stream, or synchronised).
#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/ckfwi.h"
#include "codec_common.cuh"

using namespace ckfwi;

namespace {

constexpr long long NOALLOC_MAX_BLOCKS = 65536;            // 4^d blocks per field
// the compression scratch of the largest field accepted: its layout for the
// most chunks, in 3D (a 2D chunk needs fewer staging words)
constexpr long long NOALLOC_MAX_CHUNKS = (NOALLOC_MAX_BLOCKS + CHUNK - 1) / CHUNK;
constexpr long long NOALLOC_SCRATCH_WORDS = scratch_layout_for(3, NOALLOC_MAX_CHUNKS).words;
static_assert(scratch_layout_for(2, NOALLOC_MAX_CHUNKS).words <= NOALLOC_SCRATCH_WORDS,
              "a 2D field of the largest size must fit the static scratch");

// Device-side scratch.  In host code these names are host-side stand-ins,
// not device addresses: the address is looked up once per device below.
static __device__ __align__(256) uint32_t g_scratch[NOALLOC_SCRATCH_WORDS];
static __device__ __align__(256) long long g_scalars[8];    // base, next, pad, pad, error bits

constexpr int MAX_DEV = 64;
std::mutex g_mu;
void* g_scratch_addr[MAX_DEV] = {};
void* g_scalars_addr[MAX_DEV] = {};

// Resolve the device addresses of the two arrays for the current device
// (once per device, on that device's first call).
int resolve(int dev, uint32_t** scratch, long long** scalars)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* a = nullptr;
        void* b = nullptr;
        if (cudaGetSymbolAddress(&a, g_scratch) != cudaSuccess) return CKFWI_ECUDA;
        if (cudaGetSymbolAddress(&b, g_scalars) != cudaSuccess) return CKFWI_ECUDA;
        g_scratch_addr[dev] = a;
        g_scalars_addr[dev] = b;
    }
    *scratch = static_cast<uint32_t*>(g_scratch_addr[dev]);
    *scalars = static_cast<long long*>(g_scalars_addr[dev]);
    return CKFWI_OK;
}

}  // namespace

extern "C" int ckfwi_codec_compress_noalloc(const float* x, int dims, int nz, int ny, int nx, double tol,
                                            uint32_t* out, long long cap, long long* used_words, int* flags,
                                            void* stream)
{
    if (!x || !out || cap <= 0) return CKFWI_EINVAL;
    if ((dims != 2 && dims != 3) || nz < 1 || ny < 1 || nx < 1 || (dims == 2 && ny != 1)) return CKFWI_EINVAL;
    if (!(tol >= std::ldexp(1.0, -90)) || !std::isfinite(tol)) return CKFWI_EINVAL;
    const long long nb = (long long)((nz + 3) / 4) * (dims == 3 ? (ny + 3) / 4 : 1) * ((nx + 3) / 4);
    if (nb > NOALLOC_MAX_BLOCKS) return CKFWI_EINVAL;     // beyond the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CKFWI_ECUDA;
    if (dev < 0 || dev >= MAX_DEV) return CKFWI_EINVAL;
    uint32_t* scratch = nullptr;
    long long* sc = nullptr;
    const int rs = resolve(dev, &scratch, &sc);
    if (rs != CKFWI_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (codec_scratch_bytes(dims, nz, ny, nx) > (long long)sizeof(uint32_t) * NOALLOC_SCRATCH_WORDS)
        return CKFWI_EINVAL;
    // the stream's start word, end word and error bits start at zero, and
    // so do the scratch's counter and group sums for this field's layout
    // (every other scratch word is written before it is read)
    if (cudaMemsetAsync(sc, 0, sizeof(long long) * 8, st) != cudaSuccess) return CKFWI_ECUDA;
    if (cudaMemsetAsync(scratch, 0, (size_t)codec_scratch_zero_bytes(dims, nz, ny, nx), st) != cudaSuccess)
        return CKFWI_ECUDA;
    CodecView v{};
    v.dims = dims; v.nz = nz; v.ny = ny; v.nx = nx;
    v.py = nx;
    v.pz = (long long)ny * nx;
    v.aligned = (nx % 4 == 0) && ((reinterpret_cast<uintptr_t>(x) & 15) == 0);
    float tf = (float)tol;
    if ((double)tf > tol) tf = std::nextafter(tf, 0.0f);
    int* err = reinterpret_cast<int*>(sc + 4);
    if (codec_compress_dev(x, v, tf, out, sc, cap, sc + 1, scratch, err, nullptr, st) != cudaSuccess)
        return CKFWI_ECUDA;
    long long h[5];
    if (cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return CKFWI_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CKFWI_ECUDA;
    const int e = (int)(h[4] & 0xffffffff);
    if (flags) *flags = (e & 1) ? 1 : 0;
    if (e & 2) return CKFWI_POOL_OVERFLOW;
    if (e & 4) return CKFWI_CORRUPT;          // a chunk the compaction refused: the stream is incomplete
    if (used_words) *used_words = h[1];
    return CKFWI_OK;
}
