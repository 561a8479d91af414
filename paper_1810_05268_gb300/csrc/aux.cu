// Small kernels around the time loop: receiver sampling, residual and FP64
// misfit (Sec. 6: phi = 1/2 ||d_sim - d_obs||^2), model setup (m = 1/c^2 ->
// w = dt^2 c^2), gradient output and checkpoint up-casts.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

#include "internal.h"

namespace ckfwi {

namespace {

__global__ void sample_kernel(const float* __restrict__ u, Sample smp)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= smp.n) return;
    float acc = 0.0f;
    for (int i = 0; i < smp.nst; ++i)
        acc = __fmaf_rn(smp.wt[r * smp.nst + i], __ldg(u + smp.idx[r * smp.nst + i]), acc);
    smp.out[r] = acc;
}

constexpr int RED_THREADS = 256;

// r = d - dobs for rows 1..rows-1 (row 0 zero); per-CTA FP64 partial sums
// of r^2 over a fixed contiguous range, reduced by a fixed tree.
__global__ void residual_kernel(const float* __restrict__ d, const float* __restrict__ dobs,
                                float* __restrict__ r, long long n, long long first,
                                double* __restrict__ partials, long long per_cta)
{
    __shared__ double sh[RED_THREADS];
    const long long lo = (long long)blockIdx.x * per_cta;
    const long long hi = min(lo + per_cta, n);
    double acc = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += RED_THREADS) {
        float v = 0.0f;
        double dv = 0.0;
        if (i >= first) {
            dv = (double)d[i] - (double)dobs[i];
            v = (float)dv;
        }
        r[i] = v;
        acc += dv * dv;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void final_sum_kernel(const double* __restrict__ partials, int n, double* phi)
{
    __shared__ double sh[RED_THREADS];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += RED_THREADS) acc += partials[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *phi = 0.5 * sh[0];
}

__device__ __forceinline__ long long padded(const FieldGeom& g, long long p)
{
    const long long x = p % g.nx;
    const long long t = p / g.nx;
    const long long y = t % g.ny;
    const long long z = t / g.ny;
    return z * g.pxy + y * g.px + x;
}

// kind 0: velocity c, kind 1: m = 1/c^2.  w = dt^2 c^2 (FP64, rounded once);
// c_dense keeps c in float for the gradient output.
__global__ void model_kernel(const float* __restrict__ in, int kind, double dt2, FieldGeom g,
                             float* __restrict__ w, float* __restrict__ c_dense, int* err)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.npts) return;
    const float v = in[p];
    if (!isfinite(v)) { atomicOr(err, 2); return; }
    if (!(v > 0.0f)) { atomicOr(err, 1); return; }
    double c2 = (kind == 0) ? (double)v * (double)v : 1.0 / (double)v;
    w[padded(g, p)] = (float)(dt2 * c2);
    c_dense[p] = (float)sqrt(c2);
}

// dphi/dm = gacc c^2 ; dphi/dc = dphi/dm dm/dc = -2 gacc / c
__device__ __forceinline__ float grad_value(float ga, float c, int kind)
{
    return (kind == 1) ? __fmul_rn(ga, __fmul_rn(c, c)) : __fdiv_rn(__fmul_rn(-2.0f, ga), c);
}

__global__ void grad_out_kernel(const float* __restrict__ gacc, const float* __restrict__ c,
                                int kind, float scale, FieldGeom g, float* __restrict__ out)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.npts) return;
    const float v = grad_value(gacc[padded(g, p)], c[p], kind);
    out[p] = scale == 1.0f ? v : __fmul_rn(scale, v);
}

// Neumaier-compensated FP64 accumulation of one shot's gradient into a
// dense array that may be larger than the shot's grid: point (z, y, x) of
// the grid adds into q = o0 + z * gsz + y * gsy + x.
__global__ void grad_sum_kernel(const float* __restrict__ gacc, const float* __restrict__ c,
                                int kind, FieldGeom g, long long o0, long long gsy, long long gsz,
                                double* __restrict__ sum, double* __restrict__ comp)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.npts) return;
    const long long x = p % g.nx, y = (p / g.nx) % g.ny, z = p / ((long long)g.nx * g.ny);
    const long long q = o0 + z * gsz + y * gsy + x;
    const double v = (double)grad_value(gacc[padded(g, p)], c[p], kind);
    const double s = sum[q];
    const double t = s + v;
    comp[q] += (fabs(s) >= fabs(v)) ? (s - t) + v : (v - t) + s;
    sum[q] = t;
}

// Up-cast of a checkpoint field into an FP32 working field: one thread per
// four consecutive x points of a row (one 8- or 16-byte load and one 16-byte
// store; rows start 16-byte aligned in both layouts), the ragged end of a
// row value by value.  Halo cells are not touched.
template <class T>
__device__ __forceinline__ float up1(T v);
template <> __device__ __forceinline__ float up1<float>(float v) { return v; }
template <> __device__ __forceinline__ float up1<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float up1<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class T>
__global__ void upcast_kernel(const T* __restrict__ src, FieldGeom g, float* __restrict__ dst)
{
    const long long nvx = (g.nx + 3) / 4;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nvx * g.ny * g.nz) return;
    const long long row = t / nvx;
    const int x0 = (int)(t - row * nvx) * 4;
    const long long y = row % g.ny, z = row / g.ny;
    const long long o = z * g.pxy + y * g.px + x0;
    if (x0 + 4 <= g.nx) {
        float4 r;
        if constexpr (sizeof(T) == 4) {
            r = __ldg(reinterpret_cast<const float4*>(src + o));
        } else {
            const uint2 w = __ldg(reinterpret_cast<const uint2*>(src + o));
            const T* h = reinterpret_cast<const T*>(&w);
            r = make_float4(up1<T>(h[0]), up1<T>(h[1]), up1<T>(h[2]), up1<T>(h[3]));
        }
        *reinterpret_cast<float4*>(dst + o) = r;
    } else {
        for (int i = 0; x0 + i < g.nx; ++i) dst[o + i] = up1<T>(src[o + i]);
    }
}

__global__ void copy_f64_kernel(const double* __restrict__ a, double* __restrict__ b, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

__global__ void add_f64_kernel(const double* __restrict__ a, const double* __restrict__ b, double scale,
                               double* __restrict__ out, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = scale * (a[i] + b[i]);
}

__global__ void f64_to_f32_kernel(const double* __restrict__ a, float* __restrict__ out, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)a[i];
}

// max |u| over the total grid of a padded field (the wavefield's scale, for
// stating a codec tolerance relative to it): a CTA per group of rows (z, y),
// its threads along x; the magnitudes' bit patterns order like the values,
// so one unsigned atomicMax per warp.
__global__ void absmax_kernel(const float* __restrict__ u, FieldGeom g, unsigned* __restrict__ out)
{
    unsigned m = 0u;
    const long long rows = (long long)g.nz * g.ny;
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        const long long z = r / g.ny, y = r % g.ny;
        const float* row = u + z * g.pxy + y * g.px;
        for (int x = threadIdx.x; x < g.nx; x += blockDim.x) m = max(m, __float_as_uint(fabsf(__ldg(row + x))));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_sample(const float* u, const Sample& smp, cudaStream_t s)
{
    if (smp.n <= 0) return cudaSuccess;
    sample_kernel<<<blocks_for(smp.n, 128), 128, 0, s>>>(u, smp);
    return cudaGetLastError();
}

cudaError_t launch_absmax(const float* u_origin, const FieldGeom& g, unsigned* out, cudaStream_t s)
{
    // at most 8 CTAs per SM of a 152-SM GPU, each taking rows in turn
    const unsigned nb = (unsigned)std::min<long long>((long long)g.nz * g.ny, 8LL * 152);
    absmax_kernel<<<nb, 256, 0, s>>>(u_origin, g, out);
    return cudaGetLastError();
}

cudaError_t launch_residual(const float* d, const float* dobs, float* r, int rows, int nrec,
                            double* partials, int nparts, double* phi, cudaStream_t s)
{
    const long long n = (long long)rows * nrec;
    const long long per = (n + nparts - 1) / nparts;
    residual_kernel<<<nparts, RED_THREADS, 0, s>>>(d, dobs, r, n, (long long)nrec, partials, per);
    final_sum_kernel<<<1, RED_THREADS, 0, s>>>(partials, nparts, phi);
    return cudaGetLastError();
}

cudaError_t launch_to_padded_w(const float* dense, int kind, float dt, const FieldGeom& g,
                               float* w_origin, float* c_dense, int* err, cudaStream_t s)
{
    model_kernel<<<blocks_for(g.npts, 256), 256, 0, s>>>(dense, kind, (double)dt * (double)dt, g,
                                                          w_origin, c_dense, err);
    return cudaGetLastError();
}

cudaError_t launch_grad_out(const float* gacc_origin, const float* c_dense, int kind, float scale,
                            const FieldGeom& g, float* out_dense, cudaStream_t s)
{
    grad_out_kernel<<<blocks_for(g.npts, 256), 256, 0, s>>>(gacc_origin, c_dense, kind, scale, g, out_dense);
    return cudaGetLastError();
}

cudaError_t launch_grad_out_f64(const float* gacc_origin, const float* c_dense, int kind,
                                const FieldGeom& g, long long o0, long long gsy, long long gsz,
                                double* sum, double* comp, cudaStream_t s)
{
    grad_sum_kernel<<<blocks_for(g.npts, 256), 256, 0, s>>>(gacc_origin, c_dense, kind, g, o0, gsy, gsz, sum,
                                                            comp);
    return cudaGetLastError();
}

cudaError_t launch_cast_restore(const void* src, int utype, const FieldGeom& g, float* dst_origin,
                                cudaStream_t s)
{
    const unsigned nb = blocks_for((long long)((g.nx + 3) / 4) * g.ny * g.nz, 256);
    if (utype == U_BF16)
        upcast_kernel<__nv_bfloat16><<<nb, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(src), g, dst_origin);
    else if (utype == U_FP16)
        upcast_kernel<__half><<<nb, 256, 0, s>>>(static_cast<const __half*>(src), g, dst_origin);
    else
        upcast_kernel<float><<<nb, 256, 0, s>>>(static_cast<const float*>(src), g, dst_origin);
    return cudaGetLastError();
}

cudaError_t launch_copy_f64(const double* a, double* b, long long n, cudaStream_t s)
{
    copy_f64_kernel<<<blocks_for(n, 256), 256, 0, s>>>(a, b, n);
    return cudaGetLastError();
}

}  // namespace ckfwi

namespace ckfwi {
cudaError_t launch_add_f64(const double* a, const double* b, double scale, double* out, long long n, cudaStream_t s)
{
    add_f64_kernel<<<blocks_for(n, 256), 256, 0, s>>>(a, b, scale, out, n);
    return cudaGetLastError();
}

cudaError_t launch_f64_to_f32(const double* a, float* out, long long n, cudaStream_t s)
{
    f64_to_f32_kernel<<<blocks_for(n, 256), 256, 0, s>>>(a, out, n);
    return cudaGetLastError();
}
}  // namespace ckfwi
