// The OT4 kernel: the acoustic step of fourth order in time (Sec. 6, the
// kernel the paper takes from its DSL beside OT2).  Its recursion is the OT2
// one with lap replaced by
//     A f = lap f + dt^2/12 lap(c^2 lap f)
// (the modified-equation correction of the leapfrog's dt^2/12 f_tttt error;
// include/ckfwi.h states the recursion, its adjoint and the exact gradient).
//
// A step is two launches.  The first stages f plane by plane like the OT2
// kernels and writes Z = w lap f (w = dt^2 c^2); the second applies the
// Laplacian to Z, so that
//     w A f = Z + w lap(Z) / 12,
// and finishes the leapfrog update.  Z is a full padded field whose halo
// cells are never written, so the outer Laplacian reads zeros outside the
// grid exactly as the inner one does.  Computing the inner Laplacian over a
// K-wide ring around every CTA instead would save Z's write and read but
// repeat about 1.9 times the inner stencil work at 32 x 8 tiles, and the
// step is bound by memory traffic, not by arithmetic.
//
// The reverse step needs the exact gradient's extra term
// dt^2/12 c^4 lap u^n lap lam^n.  lap lam^n needs lam^n's neighbours, which
// exist only after the step that makes lam^n, when u^n is no longer at hand.
// So each reverse step j keeps Z_u = w lap u^{j-1} for the next one, which
// pairs it with lap lam^{j-1} (both per point).  A reverse step is three
// passes, each staging at most two fields:
//   pass 1: Z_l = w lap lam^j,  Z_u(j) = w lap u^{j-1},
//           gacc += Z_u(j+1) lap(lam^j)/12                       (j < N)
//   pass 2: lam^{j-1} = leapfrog(lam^j, lam^{j+1}, Z_l + w (lap(Z_l)/12 - P^T r^j))
//           (the forward update kernel with the adjoint's fields)
//   pass 3: gacc += lam^{j-1} (lap u^{j-1} + lap(Z_u(j))/12 + q^{j-1})
// and gacc times c^2 is the gradient, as for OT2.  (Z_u(N+1) would pair with
// lap lam^N = 0; at j = 1 the term for n = 0 vanishes since u^0 = 0.)  The
// three passes move 72 B/pt against 60 for a two-pass form whose second pass
// staged all four fields, yet run 20% faster (205 against 254 us at 208^3,
// order 8): that pass needed 228 registers at two points per thread, one
// 256-thread CTA per SM.
//
// Every step of one model runs these kernels, forward and reverse, so a
// recomputed forward step repeats the first sweep bit for bit.
#include "stencil_body.cuh"

namespace ckfwi {

// One leapfrog update of the OT4 kernel, in the increment form of the OT2
// update (stencil_body.cuh):  u' = c + ((1 - e)(c - p) + Z + w s) / (1 + e),
// with Z = w lap c and s = lap(Z)/12 + sources.
__device__ __forceinline__ float leapfrog4(float c, float p, float w, float zc, float s, float eta, float hdt)
{
    const float be = __fmaf_rn(-eta, hdt, 1.0f);
    float t = __fmaf_rn(w, s, __fadd_rn(zc, __fmul_rn(be, __fsub_rn(c, p))));
    t = eta != 0.0f ? __fdividef(t, __fmaf_rn(eta, hdt, 1.0f)) : t;
    return __fadd_rn(c, t);
}

// Position of a thread's column in the step's grid.
struct Col4 {
    int tx, ty, x, y, nx, ny, nz;
    long long px, pxy, col;
    bool act;
};

// One field staged plane by plane down a CTA's z run: z neighbours in a
// register queue, the plane's x / y halos loaded one plane ahead.
template <int K, int DIMS, int BX, int BY>
struct Stage4 {
    float q[2 * K + 1];
    float nq;
    Halo<K, DIMS, BX, BY> hn, hc;

    template <class T>
    __device__ __forceinline__ void start(const T* f, const Col4& c, int z0)
    {
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) q[i] = c.act ? ldf<T>(f + (long long)(z0 - K + i) * c.pxy + c.col) : 0.0f;
        nq = c.act ? ldf<T>(f + (long long)(z0 + K) * c.pxy + c.col) : 0.0f;
        hn.load(f, (long long)z0 * c.pxy, c.col, c.tx, c.ty, c.x, c.y, c.nx, c.ny, c.px);
    }
    __device__ __forceinline__ void take()
    {
        q[2 * K] = nq;
        hc = hn;
    }
    template <class T>
    __device__ __forceinline__ void ahead(const T* f, const Col4& c, int zn)
    {
        const long long zo = (long long)zn * c.pxy;
        nq = c.act ? ldf<T>(f + zo + (long long)K * c.pxy + c.col) : 0.0f;
        hn.load(f, zo, c.col, c.tx, c.ty, c.x, c.y, c.nx, c.ny, c.px);
    }
    __device__ __forceinline__ void put(float* sm, const Col4& c) const { hc.store(sm, q[K], c.tx, c.ty); }
    __device__ __forceinline__ void shift()
    {
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) q[i] = q[i + 1];
    }
};

template <int DIMS, int BX, int BY>
__device__ __forceinline__ Col4 col4(const FieldGeom& g)
{
    Col4 c;
    c.tx = threadIdx.x;
    c.ty = threadIdx.y;
    c.nz = g.nz;
    c.ny = g.ny;
    c.nx = g.nx;
    c.px = g.px;
    c.pxy = g.pxy;
    c.x = blockIdx.x * BX + c.tx;
    c.y = (DIMS == 3) ? blockIdx.y * BY + c.ty : 0;
    c.act = (c.x < c.nx) && (c.y < c.ny);
    c.col = (long long)c.y * c.px + c.x;
    return c;
}

// ------------------------------------------------------------- pass 1
// Z_i = w lap f_i for one field (forward) or two (reverse: lam^j and u^{j-1});
// the forward pass also samples the receivers of u^n.
template <int K, int DIMS, int BX, int BY, int NF, class UT>
__global__ void __launch_bounds__(BX * BY) ot4_lap_kernel(const Ot4LapArgs a)
{
    extern __shared__ float sm[];
    constexpr int SX = BX + 2 * K;
    constexpr int TILE = (DIMS == 3 ? BY + 2 * K : 1) * SX;
    const Col4 c = col4<DIMS, BX, BY>(a.g);

    if (a.smp.n > 0) {
        const int gt = ((blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * (BX * BY) + c.ty * BX + c.tx;
        if (gt < a.smp.n) {
            float acc = 0.0f;
            for (int i = 0; i < a.smp.nst; ++i)
                acc = __fmaf_rn(a.smp.wt[gt * a.smp.nst + i], __ldg(a.f0 + a.smp.idx[gt * a.smp.nst + i]), acc);
            a.smp.out[gt] = acc;
        }
    }

    const int z0 = blockIdx.z * a.zlen;
    if (z0 >= c.nz) return;
    const int z1 = min(z0 + a.zlen, c.nz);
    const int cy = (DIMS == 3) ? c.ty + K : 0;
    const UT* f1 = static_cast<const UT*>(a.f1);
    Stage4<K, DIMS, BX, BY> s0, s1;
    s0.start(a.f0, c, z0);
    if (NF == 2) s1.start(f1, c, z0);
    float nw = c.act ? __ldg(a.w + (long long)z0 * c.pxy + c.col) : 0.0f;
    for (int z = z0; z < z1; ++z) {
        s0.take();
        if (NF == 2) s1.take();
        const float wv = nw;
        if (z + 1 < z1) {
            s0.ahead(a.f0, c, z + 1);
            if (NF == 2) s1.ahead(f1, c, z + 1);
            nw = c.act ? __ldg(a.w + (long long)(z + 1) * c.pxy + c.col) : 0.0f;
        }
        __syncthreads();
        s0.put(sm, c);
        if (NF == 2) s1.put(sm + TILE, c);
        __syncthreads();
        if (c.act) {
            const long long o = (long long)z * c.pxy + c.col;
            a.z0[o] = __fmul_rn(wv, lap_at<K, DIMS, SX>(s0.q, sm, cy, c.tx + K, a.c));
            if (NF == 2) {
                a.z1[o] = __fmul_rn(wv, lap_at<K, DIMS, SX>(s1.q, sm + TILE, cy, c.tx + K, a.c));
                if (a.zu_next)   // the deferred gradient term of the step before: Z_u(j+1) lap(lam^j)/12
                    a.gacc[o] = __fmaf_rn(__ldg(a.zu_next + o), lap_at<K, DIMS, SX>(s0.q, sm, cy, c.tx + K, a.c12),
                                          a.gacc[o]);
            }
        }
        s0.shift();
        if (NF == 2) s1.shift();
    }
}

// ------------------------------------------------------------- pass 2, forward
template <int K, int DIMS, int BX, int BY, int CK>
__global__ void __launch_bounds__(BX * BY) ot4_fwd_kernel(const Ot4FwdArgs A)
{
    extern __shared__ float sm[];
    constexpr int SX = BX + 2 * K;
    const FwdArgs& a = A.f;
    const Col4 c = col4<DIMS, BX, BY>(a.g);
    const int z0 = blockIdx.z * a.zlen;
    if (z0 >= c.nz) return;
    const int z1 = min(z0 + a.zlen, c.nz);
    const int cy = (DIMS == 3) ? c.ty + K : 0;
    const float ecol = c.act ? ((DIMS == 3 ? a.eta[c.nz + c.y] : 0.0f) + a.eta[c.nz + c.ny + c.x]) : 0.0f;
    const InjCol ic = inj_col(a.src, c.y, c.x, c.act);

    Stage4<K, DIMS, BX, BY> sz;
    sz.start(A.z, c, z0);
    long long o1 = (long long)z0 * c.pxy + c.col;
    float nu = c.act ? __ldg(a.u + o1) : 0.0f;
    float nup = c.act ? __ldg(a.up + o1) : 0.0f;
    float nw = c.act ? __ldg(a.w + o1) : 0.0f;
    for (int z = z0; z < z1; ++z) {
        sz.take();
        const float uv = nu, upv = nup, wv = nw;
        if (z + 1 < z1) {
            sz.ahead(A.z, c, z + 1);
            o1 = (long long)(z + 1) * c.pxy + c.col;
            nu = c.act ? __ldg(a.u + o1) : 0.0f;
            nup = c.act ? __ldg(a.up + o1) : 0.0f;
            nw = c.act ? __ldg(a.w + o1) : 0.0f;
        }
        __syncthreads();
        sz.put(sm, c);
        __syncthreads();
        if (c.act) {
            float s = lap_at<K, DIMS, SX>(sz.q, sm, cy, c.tx + K, A.c12);
            s = __fadd_rn(s, inj_val(a.src, ic, z));
            const float eta = a.eta[z] + ecol;
            const float v = leapfrog4(uv, upv, wv, sz.q[K], s, eta, a.hdt);
            const long long o = (long long)z * c.pxy + c.col;
            a.out[o] = v;
            if (CK == CK_FP32) {
                static_cast<float*>(a.ck_up)[o] = uv;
            } else if (CK == CK_BF16) {
                static_cast<__nv_bfloat16*>(a.ck_u)[o] = __float2bfloat16_rn(v);
                static_cast<__nv_bfloat16*>(a.ck_up)[o] = __float2bfloat16_rn(uv);
            } else if (CK == CK_FP16) {
                const __half hv = __float2half_rn(v), hp = __float2half_rn(uv);
                static_cast<__half*>(a.ck_u)[o] = hv;
                static_cast<__half*>(a.ck_up)[o] = hp;
                if (__hisinf(hv) || __hisinf(hp)) atomicOr(a.err, 1);
            }
        }
        sz.shift();
    }
}

// ------------------------------------------------------------- pass 3, reverse
template <int K, int DIMS, int BX, int BY, class UT>
__global__ void __launch_bounds__(BX * BY) ot4_grad_kernel(const Ot4GradArgs a)
{
    extern __shared__ float sm[];
    constexpr int SX = BX + 2 * K;
    constexpr int TILE = (DIMS == 3 ? BY + 2 * K : 1) * SX;
    const Col4 c = col4<DIMS, BX, BY>(a.g);
    const int z0 = blockIdx.z * a.zlen;
    if (z0 >= c.nz) return;
    const int z1 = min(z0 + a.zlen, c.nz);
    const int cy = (DIMS == 3) ? c.ty + K : 0;
    const InjCol is = inj_col(a.src, c.y, c.x, c.act);
    const UT* uu = static_cast<const UT*>(a.u);
    float* smu = sm;
    float* smzu = sm + TILE;
    Stage4<K, DIMS, BX, BY> su, szu;
    su.start(uu, c, z0);
    szu.start(a.zu, c, z0);
    long long o1 = (long long)z0 * c.pxy + c.col;
    float nl = c.act ? __ldg(a.l0 + o1) : 0.0f;
    float ng = c.act ? a.gacc[o1] : 0.0f;
    for (int z = z0; z < z1; ++z) {
        su.take();
        szu.take();
        const float lv = nl, gv = ng;
        if (z + 1 < z1) {
            su.ahead(uu, c, z + 1);
            szu.ahead(a.zu, c, z + 1);
            o1 = (long long)(z + 1) * c.pxy + c.col;
            nl = c.act ? __ldg(a.l0 + o1) : 0.0f;
            ng = c.act ? a.gacc[o1] : 0.0f;
        }
        __syncthreads();
        su.put(smu, c);
        szu.put(smzu, c);
        __syncthreads();
        if (c.act) {
            float g = lap_at<K, DIMS, SX>(su.q, smu, cy, c.tx + K, a.c);
            g = __fadd_rn(g, lap_at<K, DIMS, SX>(szu.q, smzu, cy, c.tx + K, a.c12));
            g = __fadd_rn(g, inj_val(a.src, is, z));
            a.gacc[(long long)z * c.pxy + c.col] = __fmaf_rn(lv, g, gv);
        }
        su.shift();
        szu.shift();
    }
}

// ---------------------------------------------------------------- dispatch
namespace {
template <int DIMS, int BX, int BY>
dim3 grid_of(const FieldGeom& g, int zlen)
{
    return dim3((g.nx + BX - 1) / BX, DIMS == 3 ? (g.ny + BY - 1) / BY : 1, (g.nz + zlen - 1) / zlen);
}

template <int K, int DIMS, int BX, int BY>
cudaError_t lap_go(const Ot4LapArgs& a, int ut, cudaStream_t s)
{
    const dim3 blk(BX, BY, 1), grd = grid_of<DIMS, BX, BY>(a.g, a.zlen);
    const int nf = a.f1 ? 2 : 1;
    const size_t sh = smem_bytes<DIMS, BX, BY>(K, nf);
    if (nf == 1) {
        ot4_lap_kernel<K, DIMS, BX, BY, 1, float><<<grd, blk, sh, s>>>(a);
    } else {
        switch (ut) {
        case U_FP32: ot4_lap_kernel<K, DIMS, BX, BY, 2, float><<<grd, blk, sh, s>>>(a); break;
        case U_BF16: ot4_lap_kernel<K, DIMS, BX, BY, 2, __nv_bfloat16><<<grd, blk, sh, s>>>(a); break;
        case U_FP16: ot4_lap_kernel<K, DIMS, BX, BY, 2, __half><<<grd, blk, sh, s>>>(a); break;
        default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

template <int K, int DIMS, int BX, int BY>
cudaError_t fwd2_go(const Ot4FwdArgs& a, int ck, cudaStream_t s)
{
    const dim3 blk(BX, BY, 1), grd = grid_of<DIMS, BX, BY>(a.f.g, a.f.zlen);
    const size_t sh = smem_bytes<DIMS, BX, BY>(K, 1);
    switch (ck) {
    case CK_NONE: ot4_fwd_kernel<K, DIMS, BX, BY, CK_NONE><<<grd, blk, sh, s>>>(a); break;
    case CK_FP32: ot4_fwd_kernel<K, DIMS, BX, BY, CK_FP32><<<grd, blk, sh, s>>>(a); break;
    case CK_BF16: ot4_fwd_kernel<K, DIMS, BX, BY, CK_BF16><<<grd, blk, sh, s>>>(a); break;
    case CK_FP16: ot4_fwd_kernel<K, DIMS, BX, BY, CK_FP16><<<grd, blk, sh, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int K, int DIMS, int BX, int BY>
cudaError_t grad_go(const Ot4GradArgs& a, int ut, cudaStream_t s)
{
    const dim3 blk(BX, BY, 1), grd = grid_of<DIMS, BX, BY>(a.g, a.zlen);
    const size_t sh = smem_bytes<DIMS, BX, BY>(K, 2);
    switch (ut) {
    case U_FP32: ot4_grad_kernel<K, DIMS, BX, BY, float><<<grd, blk, sh, s>>>(a); break;
    case U_BF16: ot4_grad_kernel<K, DIMS, BX, BY, __nv_bfloat16><<<grd, blk, sh, s>>>(a); break;
    case U_FP16: ot4_grad_kernel<K, DIMS, BX, BY, __half><<<grd, blk, sh, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// tile shapes: 3D 32 x 8 and 32 x 16 (rows >= K for the y halo), 2D 128 points
template <int K, class F3a, class F3b, class F2>
cudaError_t by_shape(int dims, const Tile& t, F3a f3a, F3b f3b, F2 f2)
{
    if (dims == 3) {
        if (t.bx == 32 && t.by == 8) return f3a();
        if (t.bx == 32 && t.by == 16) return f3b();
    } else if (t.bx == 128) {
        return f2();
    }
    return cudaErrorInvalidValue;
}

template <int K>
cudaError_t lap_k(const Ot4LapArgs& a, const Tile& t, int ut, cudaStream_t s)
{
    return by_shape<K>(
        a.g.dims, t, [&] { return lap_go<K, 3, 32, 8>(a, ut, s); }, [&] { return lap_go<K, 3, 32, 16>(a, ut, s); },
        [&] { return lap_go<K, 2, 128, 1>(a, ut, s); });
}

template <int K>
cudaError_t fwd2_k(const Ot4FwdArgs& a, const Tile& t, int ck, cudaStream_t s)
{
    return by_shape<K>(
        a.f.g.dims, t, [&] { return fwd2_go<K, 3, 32, 8>(a, ck, s); },
        [&] { return fwd2_go<K, 3, 32, 16>(a, ck, s); }, [&] { return fwd2_go<K, 2, 128, 1>(a, ck, s); });
}

template <int K>
cudaError_t grad_k(const Ot4GradArgs& a, const Tile& t, int ut, cudaStream_t s)
{
    return by_shape<K>(
        a.g.dims, t, [&] { return grad_go<K, 3, 32, 8>(a, ut, s); },
        [&] { return grad_go<K, 3, 32, 16>(a, ut, s); }, [&] { return grad_go<K, 2, 128, 1>(a, ut, s); });
}
}  // namespace

bool ot4_supported(int dims, int K, const Tile& t)
{
    if (t.ver != 5 || t.zlen < 1) return false;
    if (K != 1 && K != 2 && K != 4 && K != 8) return false;
    if (dims == 3) return t.bx == 32 && (t.by == 8 || t.by == 16) && t.by >= K;
    return t.bx == 128 && t.by == 1;
}

int ot4_shape_count(int dims) { return dims == 3 ? 2 : 1; }

Tile ot4_tile_at(int dims, int i, int zlen)
{
    Tile t;
    t.ver = 5;
    t.bx = dims == 3 ? 32 : 128;
    t.by = dims == 3 ? (i == 0 ? 8 : 16) : 1;
    t.zlen = zlen;
    return t;
}

cudaError_t launch_ot4_lap(const Ot4LapArgs& a, const Tile& t, int K, int ut, cudaStream_t s)
{
    Ot4LapArgs b = a;
    b.zlen = t.zlen;
    switch (K) {
    case 1: return lap_k<1>(b, t, ut, s);
    case 2: return lap_k<2>(b, t, ut, s);
    case 4: return lap_k<4>(b, t, ut, s);
    case 8: return lap_k<8>(b, t, ut, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ot4_fwd(const Ot4FwdArgs& a, const Tile& t, int K, int ck, cudaStream_t s)
{
    Ot4FwdArgs b = a;
    b.f.zlen = t.zlen;
    switch (K) {
    case 1: return fwd2_k<1>(b, t, ck, s);
    case 2: return fwd2_k<2>(b, t, ck, s);
    case 4: return fwd2_k<4>(b, t, ck, s);
    case 8: return fwd2_k<8>(b, t, ck, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ot4_grad(const Ot4GradArgs& a, const Tile& t, int K, int ut, cudaStream_t s)
{
    Ot4GradArgs b = a;
    b.zlen = t.zlen;
    switch (K) {
    case 1: return grad_k<1>(b, t, ut, s);
    case 2: return grad_k<2>(b, t, ut, s);
    case 4: return grad_k<4>(b, t, ut, s);
    case 8: return grad_k<8>(b, t, ut, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ckfwi
