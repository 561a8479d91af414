// C-ABI of the ckfwi library: model set-up, forward modelling, and the
// checkpointed (optionally compressed) adjoint-state gradient executor.
//
// The executor walks the Revolve action list (Sec. 3) and maps every action
// to kernel launches on the caller's stream:
//   advance(s, k)  k forward steps; in the first sweep each step also
//                  samples the receivers; the step that ends on a state
//                  about to be stored writes the checkpoint itself (fused
//                  takeshot: FP32 writes u^{n+1} straight into the slot and
//                  copies u^n beside it, BF16 / FP16 write both casts)
//   takeshot(s)    fused as above, or two codec compressions (Sec. 4)
//   restore(s)     FP32: the slot becomes the current state (no copy);
//                  BF16 / FP16 / codec: up-cast or decode into working
//                  fields -- only u^s when the next action is a reverse step
//   youturn(s)     one fused reverse step (adjoint + imaging condition)
// Before the first reverse step the state N-1 is advanced once more to
// record d^{N-1} and d^N, and the residual and FP64 misfit are formed on the
// device.  Nothing synchronises with the host until the gradient is done.
// With M >= N every state is kept instead (store-all): the forward sweep
// writes u^{n+1} straight into the trajectory.
// Every action is an NVTX range named after it ("ckfwi advance" and so on,
// the state as payload) inside a "ckfwi gradient" range; with use_graph the
// ranges mark the recording call only.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <set>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ckfwi.h"
#include "internal.h"
#include "revolve.h"

using namespace ckfwi;

namespace {

#define CK_TRY(expr)                                   \
    do {                                               \
        cudaError_t e_ = (expr);                       \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

#define ST_TRY(expr)                 \
    do {                             \
        int s_ = (expr);             \
        if (s_ != CKFWI_OK) return s_; \
    } while (0)

int cuda_status(cudaError_t e)
{
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return CKFWI_ENOMEM;
    }
    return CKFWI_ECUDA;
}

int cuda_status_or_ok(cudaError_t e) { return e == cudaSuccess ? CKFWI_OK : cuda_status(e); }

struct DevMem {
    void* p = nullptr;
    size_t bytes = 0;
    DevMem() = default;
    DevMem(const DevMem&) = delete;
    DevMem& operator=(const DevMem&) = delete;
    ~DevMem() { release(); }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    // (Re)allocate when too small.  A fresh allocation is zeroed when asked
    // (the zero halo cells of a field must hold 0 and are never written); a
    // reused one keeps its contents.
    cudaError_t alloc(size_t n, bool zero = true)
    {
        if (bytes >= n && p) return cudaSuccess;
        release();
        if (n == 0) return cudaSuccess;
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = n;
        if (zero) {
            e = cudaMemset(p, 0, n);
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
        }
        return e;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// Pinned, device-mapped host memory (the second checkpoint level).
struct HostMem {
    void* p = nullptr;     // host address
    void* d = nullptr;     // the device's address of the same bytes
    size_t bytes = 0;
    HostMem() = default;
    HostMem(const HostMem&) = delete;
    HostMem& operator=(const HostMem&) = delete;
    ~HostMem() { release(); }
    void release()
    {
        if (p) cudaFreeHost(p);
        p = d = nullptr;
        bytes = 0;
    }
    // (re)allocate when too small; a fresh allocation is zeroed
    cudaError_t alloc(size_t n)
    {
        if (bytes >= n && p) return cudaSuccess;
        release();
        if (n == 0) return cudaSuccess;
        cudaError_t e = cudaHostAlloc(&p, n, cudaHostAllocMapped | cudaHostAllocPortable);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        std::memset(p, 0, n);
        e = cudaHostGetDevicePointer(&d, p, 0);
        if (e != cudaSuccess) {
            release();
            return e;
        }
        bytes = n;
        return cudaSuccess;
    }
};


// FD weights of the 2k-th order second derivative, closed form (k! )^2 ...
void fd_weights(int k, double* c)
{
    double kf = 1.0;
    for (int i = 2; i <= k; ++i) kf *= i;
    double sum = 0.0;
    for (int j = 1; j <= k; ++j) {
        double a = 1.0, b = 1.0;
        for (int i = 2; i <= k - j; ++i) a *= i;
        for (int i = 2; i <= k + j; ++i) b *= i;
        double cj = 2.0 * kf * kf / ((double)j * j * a * b);
        c[j] = (j % 2 == 1) ? cj : -cj;
        sum += c[j];
    }
    c[0] = -2.0 * sum;
}

// Multilinear stencil of a position [m] (from the first interior point).
// Per axis: grid coordinate gc = nbl + pos/h must lie in [0, n-1];
// base i0 = min(floor(gc), n-2), fraction gc - i0.
bool interp_stencil(const ckfwi_grid& g, const double* pos, int idx3[8][3], double wt[8], int* cnt)
{
    const int ns[3] = {g.n[0], g.n[1], g.n[2]};
    int i0[3] = {0, 0, 0};
    double fr[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        if (a == 1 && g.dims == 2) continue;
        const double gc = g.nbl + pos[a] / g.h;
        if (!(gc >= 0.0) || gc > (double)(ns[a] - 1)) return false;
        int b = (int)std::floor(gc);
        if (b > ns[a] - 2) b = ns[a] - 2;
        i0[a] = b;
        fr[a] = gc - b;
    }
    int k = 0;
    const int ny = g.dims == 3 ? 2 : 1;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < ny; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = (dz ? fr[0] : 1 - fr[0]) * (dx ? fr[2] : 1 - fr[2]);
                if (g.dims == 3) w *= dy ? fr[1] : 1 - fr[1];
                idx3[k][0] = i0[0] + dz;
                idx3[k][1] = g.dims == 3 ? i0[1] + dy : 0;
                idx3[k][2] = i0[2] + dx;
                wt[k] = w;
                ++k;
            }
    *cnt = k;
    return true;
}

// Host-built CSR gather over the bounding box of a set of weighted points.
struct HostInj {
    int z0 = 0, z1 = 0, y0 = 0, y1 = 0, x0 = 0, x1 = 0;
    std::vector<int> rowptr, col;
    std::vector<float> wt;
};

struct Entry {
    int z, y, x, col;
    double w;
};

HostInj build_inj(std::vector<Entry> es)
{
    HostInj h;
    if (es.empty()) return h;
    h.z0 = h.z1 = es[0].z;
    h.y0 = h.y1 = es[0].y;
    h.x0 = h.x1 = es[0].x;
    for (auto& e : es) {
        h.z0 = std::min(h.z0, e.z); h.z1 = std::max(h.z1, e.z);
        h.y0 = std::min(h.y0, e.y); h.y1 = std::max(h.y1, e.y);
        h.x0 = std::min(h.x0, e.x); h.x1 = std::max(h.x1, e.x);
    }
    h.z1 += 1; h.y1 += 1; h.x1 += 1;
    const long long by = h.y1 - h.y0, bx = h.x1 - h.x0;
    const long long nb = (long long)(h.z1 - h.z0) * by * bx;
    auto key = [&](const Entry& e) { return ((long long)(e.z - h.z0) * by + (e.y - h.y0)) * bx + (e.x - h.x0); };
    std::stable_sort(es.begin(), es.end(), [&](const Entry& a, const Entry& b) {
        const long long ka = key(a), kb = key(b);
        return ka != kb ? ka < kb : a.col < b.col;
    });
    h.rowptr.assign(nb + 1, 0);
    for (auto& e : es) h.rowptr[key(e) + 1]++;
    for (long long i = 0; i < nb; ++i) h.rowptr[i + 1] += h.rowptr[i];
    for (auto& e : es) {
        h.col.push_back(e.col);
        h.wt.push_back((float)e.w);
    }
    return h;
}

struct DevInj {
    DevMem rowptr, col, wt;
    Inj view{};   // series filled per launch
    int set(const HostInj& h)
    {
        view = Inj{};
        if (h.rowptr.empty()) return CKFWI_OK;
        CK_TRY(rowptr.alloc(h.rowptr.size() * sizeof(int), false));
        CK_TRY(col.alloc(std::max<size_t>(1, h.col.size()) * sizeof(int), false));
        CK_TRY(wt.alloc(std::max<size_t>(1, h.wt.size()) * sizeof(float), false));
        CK_TRY(cudaMemcpy(rowptr.p, h.rowptr.data(), h.rowptr.size() * sizeof(int), cudaMemcpyHostToDevice));
        if (!h.col.empty()) {
            CK_TRY(cudaMemcpy(col.p, h.col.data(), h.col.size() * sizeof(int), cudaMemcpyHostToDevice));
            CK_TRY(cudaMemcpy(wt.p, h.wt.data(), h.wt.size() * sizeof(float), cudaMemcpyHostToDevice));
        }
        view.on = 1;
        view.z0 = h.z0; view.z1 = h.z1; view.y0 = h.y0; view.y1 = h.y1; view.x0 = h.x0; view.x1 = h.x1;
        view.rowptr = rowptr.as<int>();
        view.col = col.as<int>();
        view.wt = wt.as<float>();
        return CKFWI_OK;
    }
};

// geometry of one shot on the device
struct ShotDev {
    int nrec = 0;
    int nst = 0;
    DevMem ridx, rwt, wavelet;
    DevInj src, adj;
    DevMem dsim, dobs, resid;
    std::vector<unsigned char> key;    // host description the maps were built from
};

struct GraphKey {
    int nt, M, mode, kind;
    float tol;
    size_t pool;
    long long gen;      // buffer generation the graph's pointers belong to
    bool operator<(const GraphKey& o) const
    {
        return std::tie(nt, M, mode, kind, tol, pool, gen) <
               std::tie(o.nt, o.M, o.mode, o.kind, o.tol, o.pool, o.gen);
    }
};

// An instantiated graph and what its recording launched.
struct GraphExec {
    cudaGraphExec_t ex = nullptr;
    long long launches = 0;
    long long count[5] = {0, 0, 0, 0, 0};
    GraphExec() = default;
    GraphExec(const GraphExec&) = delete;
    GraphExec& operator=(const GraphExec&) = delete;
    ~GraphExec() { release(); }
    void release()
    {
        if (ex) cudaGraphExecDestroy(ex);
        ex = nullptr;
    }
};

constexpr size_t MAX_GRAPHS = 8;   // recorded graphs kept per model

// Tile shape and per-lane z-run lengths of a batch of lanes.
struct BatchTiles {
    Tile tf{}, ta{};
    std::vector<int> zf, za;
};

struct BatchKey {
    std::vector<long long> lanes;   // (uid, gen) of every lane
    int nt, M, mode, kind;
    float tol;
    bool operator<(const BatchKey& o) const
    {
        return std::tie(lanes, nt, M, mode, kind, tol) < std::tie(o.lanes, o.nt, o.M, o.mode, o.kind, o.tol);
    }
};

// A recorded batch and the argument tables its launches read.
struct BatchGraph {
    GraphExec ex;
    DevMem tabs;
    void release() { ex.release(); }
};

}  // namespace

struct ckfwi_model {
    ckfwi_grid g{};
    FieldGeom fg{};
    int K = 0;
    float c[MAXK + 1] = {};
    float hdt = 0.0f;
    int ot = 2;                     // time order of the kernel: 2 (OT2) or 4 (OT4)
    float c12[MAXK + 1] = {};       // OT4: c_j / (12 h^2)
    DevMem z4[3];                   // OT4: w lap f of the step in flight, and w lap u of the
                                    // last two reverse steps (alternating by step parity)
    bool have_model = false;
    DevMem eta, w, cvel, zero, uN;
    DevMem work[3], lam[3], gacc;
    DevMem traj;                    // store-all trajectory
    DevMem pool;                    // checkpoint pool
    HostMem hpool;                  // checkpoint slots in host memory (second level)
    int host_slots = 0;             // slots 1 .. host_slots live in hpool
    long long wait_limit = 1LL << 22;   // TMA kernels: back-off rounds of a plane's wait
    size_t pool_cap_bytes = 0;
    int pool_tag = -1;              // storage mode whose layout the pool holds
    DevMem slotbase;                // codec: device word offsets of slots
    DevMem scratch;                 // codec scratch
    DevMem flags;                   // int error flags
    DevMem phi, partials;
    DevMem statw;                   // codec: words per compression
    std::vector<long long> last_words;   // codec: words of each compression of the last gradient
    DevMem gsum_comp;               // batch: compensation terms
    ShotDev shot;
    Tile tf{}, ta{};
    bool tuned = false;
    int nparts = 128;
    long long gen = 0;              // bumped whenever a buffer a graph uses moves
    cudaStream_t cap = nullptr;     // non-blocking stream used only to record graphs
    cudaEvent_t ev = nullptr;
    std::vector<cudaEvent_t> evpool; // profiling events, reused across calls
    std::map<std::tuple<const void*, int, int, int>, CUtensorMap> tmaps;   // (base, dtype, box x, box y)
    long long uid = 0;              // process-unique id (batch graph keys)
    long long model_ver = 0;        // bumped by every ckfwi_set_model
    long long src_ver = -1;         // clone: the parent's model_ver its medium copies
    long long cap_words = 0;        // codec pool capacity [words]
    // graphs
    std::map<GraphKey, GraphExec> graphs;
    std::vector<GraphKey> graph_order;
    // batches of shots: clones of this model serve as extra lanes
    std::vector<std::unique_ptr<ckfwi_model>> clones;
    std::map<std::vector<long long>, BatchTiles> btiles;
    std::map<BatchKey, BatchGraph> bgraphs;
    std::vector<BatchKey> bgraph_order;
    DevMem btabs;                   // batch argument tables of an unrecorded run
    DevMem hostgrad;                // device staging of a gradient returned to host memory
    // FP32 slots in host memory, staged: a checkpoint goes to one of three
    // device staging pairs (hstage, used in turn, so the pair a step writes is
    // never one the step reads) in the step that makes it and is copied to
    // its host slot on the copy stream `side`, overlapped with the next
    // steps; a restore reads one of two device pairs (hrest), filled by a
    // copy on the copy stream as soon as the previous host restore has
    // happened (the schedule is known), or on the main stream if it could
    // not be prefetched
    DevMem hstage[3][2], hrest[2][2];
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_done[3] = {nullptr, nullptr, nullptr}, ev_pf[2] = {nullptr, nullptr},
                ev_join = nullptr;
    ~ckfwi_model()
    {
        graphs.clear();
        bgraphs.clear();
        if (side) cudaStreamDestroy(side);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        for (cudaEvent_t e : ev_done)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : ev_pf)
            if (e) cudaEventDestroy(e);
        if (cap) cudaStreamDestroy(cap);
        if (ev) cudaEventDestroy(ev);
        for (cudaEvent_t e : evpool) cudaEventDestroy(e);
    }
};

namespace ckfwi {

FieldGeom make_geom(int dims, int nz, int ny, int nx, int H)
{
    FieldGeom f{};
    f.dims = dims;
    f.nz = nz;
    f.ny = ny;
    f.nx = nx;
    f.H = H;
    f.X0 = ((H + 3) / 4) * 4;
    if (f.X0 < 4) f.X0 = 4;
    f.px = ((f.X0 + nx + H + 31) / 32) * 32;
    const long long py = dims == 3 ? ny + 2LL * H : 1;
    f.pxy = f.px * py;
    const long long pz = nz + 2LL * H;
    f.origin = (long long)H * f.pxy + (dims == 3 ? (long long)H * f.px : 0) + f.X0;
    f.alloc = pz * f.pxy + 64;
    f.npts = (long long)nz * ny * nx;
    return f;
}

}  // namespace ckfwi

namespace {

float* org(const DevMem& m, const FieldGeom& g) { return m.as<float>() + g.origin; }

size_t field_bytes(const FieldGeom& g, size_t elem = 4) { return (size_t)g.alloc * elem; }
// cuTensorMapEncodeTiled, fetched from the driver through the runtime (no
// link-time dependency on libcuda).
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn()
{
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

// Tensor map of a padded field (3D: x = px, y = ny + 2H, z = nz + 2H in
// storage coordinates), box (bx, by, 1); elem 4 = FP32, 2 = BF16 or FP16.
int tensor_map(ckfwi_model* m, const void* origin_ptr, int utype, int bx, int by, CUtensorMap* out);

double eta_axis(const ckfwi_grid& g, int i, int n)
{
    if (g.nbl <= 0) return 0.0;
    const double L = g.nbl * g.h;
    const double emax = 3.0 * g.vmax_damp / (2.0 * L) * std::log(1.0 / 1e-3);
    double delta = 0.0;
    if (i < g.nbl) delta = (double)(g.nbl - i) * g.h;
    else if (i > n - 1 - g.nbl) delta = (double)(i - (n - 1 - g.nbl)) * g.h;
    const double r = delta / L;
    return emax * r * r;
}

cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

int check_grid(const ckfwi_grid* g)
{
    if (!g) return CKFWI_EINVAL;
    if (g->dims != 2 && g->dims != 3) return CKFWI_EINVAL;
    if (g->n[0] < 2 || g->n[2] < 2) return CKFWI_EINVAL;
    if (g->dims == 2 && g->n[1] != 1) return CKFWI_EINVAL;
    if (g->dims == 3 && g->n[1] < 2) return CKFWI_EINVAL;
    const int so = g->space_order;
    if (so != 2 && so != 4 && so != 8 && so != 16) return CKFWI_EINVAL;
    if (!(g->h > 0) || !(g->dt > 0) || g->nt < 1 || g->nbl < 0) return CKFWI_EINVAL;
    if (!(g->vmax_damp > 0)) return CKFWI_EINVAL;
    if (2LL * g->nbl >= g->n[0] || 2LL * g->nbl >= g->n[2]) return CKFWI_EINVAL;
    if (g->time_order != 0 && g->time_order != 2 && g->time_order != 4) return CKFWI_EINVAL;
    // leapfrog stability: x = (vmax dt / h)^2 * dims * |symbol at k h = pi| <= 4,
    // the 1-D symbol of the 2k-th order second difference being -4 sum_{j odd} c_j.
    // OT4 multiplies a mode by 2 - x + x^2/12 per step instead of 2 - x, which
    // stays within [-2, 2] up to x = 12.
    double c[MAXK + 1];
    fd_weights(so / 2, c);
    double sym = 0.0;
    for (int j = 1; j <= so / 2; j += 2) sym += 4.0 * c[j];
    const double cfl = g->vmax_damp * g->dt / g->h;
    if (cfl * cfl * g->dims * sym > (g->time_order == 4 ? 12.0 : 4.0)) return CKFWI_EINVAL;
    return CKFWI_OK;
}

// ---------------------------------------------------------------- shots
int set_shot(ckfwi_model* m, const ckfwi_shot* s)
{
    if (!s || s->nrec < 1 || !s->rec) return CKFWI_EINVAL;
    const ckfwi_grid& g = m->g;
    // cache key: the shot description
    std::vector<unsigned char> key(sizeof(double) * 6 + sizeof(int) + sizeof(double) * 3 * s->nrec +
                                   (s->wavelet ? sizeof(float) * g.nt : 0));
    {
        unsigned char* p = key.data();
        const double hd[6] = {s->src[0], s->src[1], s->src[2], s->f0, s->t0, s->amp};
        std::memcpy(p, hd, sizeof(hd));
        p += sizeof(hd);
        std::memcpy(p, &s->nrec, sizeof(int));
        p += sizeof(int);
        std::memcpy(p, s->rec, sizeof(double) * 3 * s->nrec);
        p += sizeof(double) * 3 * s->nrec;
        if (s->wavelet) std::memcpy(p, s->wavelet, sizeof(float) * g.nt);
    }
    if (key == m->shot.key) return CKFWI_OK;
    ShotDev& d = m->shot;
    d.key.clear();
    ++m->gen;
    const FieldGeom& f = m->fg;
    int cnt = 0;
    int idx3[8][3];
    double wt[8];
    // source
    if (!interp_stencil(g, s->src, idx3, wt, &cnt)) return CKFWI_EINVAL;
    std::vector<Entry> es;
    for (int i = 0; i < cnt; ++i) es.push_back(Entry{idx3[i][0], idx3[i][1], idx3[i][2], 0, wt[i]});
    ST_TRY(d.src.set(build_inj(es)));
    std::vector<float> wav(g.nt);
    if (s->wavelet) {
        for (int n = 0; n < g.nt; ++n) {
            if (!std::isfinite(s->wavelet[n])) return CKFWI_NONFINITE;
            wav[n] = s->wavelet[n];
        }
    } else {
        if (!(s->f0 > 0)) return CKFWI_EINVAL;
        const double t0 = s->t0 > 0 ? s->t0 : 1.5 / s->f0;
        const double pi = 3.14159265358979323846;
        for (int n = 0; n < g.nt; ++n) {
            const double t = n * g.dt - t0;
            const double a = pi * pi * s->f0 * s->f0 * t * t;
            wav[n] = (float)(s->amp * (1.0 - 2.0 * a) * std::exp(-a));
        }
    }
    CK_TRY(d.wavelet.alloc(sizeof(float) * g.nt, false));
    CK_TRY(cudaMemcpy(d.wavelet.p, wav.data(), sizeof(float) * g.nt, cudaMemcpyHostToDevice));
    // receivers: sampling stencils and the adjoint-source gather (-P^T)
    const int nst = g.dims == 3 ? 8 : 4;
    std::vector<long long> ridx((size_t)s->nrec * nst);
    std::vector<float> rw((size_t)s->nrec * nst);
    es.clear();
    for (int r = 0; r < s->nrec; ++r) {
        if (!interp_stencil(g, s->rec + 3 * r, idx3, wt, &cnt)) return CKFWI_EINVAL;
        for (int i = 0; i < cnt; ++i) {
            ridx[(size_t)r * nst + i] = (long long)idx3[i][0] * f.pxy + (long long)idx3[i][1] * f.px + idx3[i][2];
            rw[(size_t)r * nst + i] = (float)wt[i];
            es.push_back(Entry{idx3[i][0], idx3[i][1], idx3[i][2], r, -wt[i]});
        }
    }
    ST_TRY(d.adj.set(build_inj(es)));
    CK_TRY(d.ridx.alloc(ridx.size() * sizeof(long long), false));
    CK_TRY(d.rwt.alloc(rw.size() * sizeof(float), false));
    CK_TRY(cudaMemcpy(d.ridx.p, ridx.data(), ridx.size() * sizeof(long long), cudaMemcpyHostToDevice));
    CK_TRY(cudaMemcpy(d.rwt.p, rw.data(), rw.size() * sizeof(float), cudaMemcpyHostToDevice));
    const size_t nd = (size_t)(g.nt + 1) * s->nrec;
    CK_TRY(d.dsim.alloc(nd * sizeof(float)));
    CK_TRY(d.dobs.alloc(nd * sizeof(float)));
    CK_TRY(d.resid.alloc(nd * sizeof(float)));
    d.nrec = s->nrec;
    d.nst = nst;
    d.key = std::move(key);
    return CKFWI_OK;
}

// ---------------------------------------------------------------- launches
enum { PC_FWD = 0, PC_ADJ = 1, PC_COMP = 2, PC_DECOMP = 3, PC_OTHER = 4, PC_N = 5 };

// Optional per-class device timing: an event pair around every launch group.
struct Prof {
    bool on = false;
    std::vector<cudaEvent_t>* pool = nullptr;
    std::vector<std::pair<int, int>> marks;   // (class, index of the start event)
    size_t next = 0;
    cudaEvent_t take()
    {
        if (next == pool->size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pool->push_back(e);
        }
        return (*pool)[next++];
    }
};

// The buffers a schedule step reads and writes.  Every lane (shot) of a
// batch runs the same schedule, so a step names roles, and each lane
// resolves them to its own buffers.
enum RoleKind { R_NONE, R_ZERO, R_WORK, R_LAM, R_UN, R_TRAJ, R_SLOT, R_HSTAGE, R_HREST };
struct Role {
    int kind = R_NONE;
    int idx = 0;      // work / lam index, trajectory level, or slot (>= 1)
    int which = 0;    // slot: 0 = u^s, 1 = u^{s-1}
    bool operator==(const Role& o) const { return kind == o.kind && idx == o.idx && which == o.which; }
    bool operator!=(const Role& o) const { return !(*this == o); }
};
const Role NONE_R{R_NONE, 0, 0};
const Role ZERO_R{R_ZERO, 0, 0};
const Role UN_R{R_UN, 0, 0};
Role work_r(int i) { return Role{R_WORK, i, 0}; }
Role lam_r(int i) { return Role{R_LAM, i, 0}; }
Role traj_r(int n) { return Role{R_TRAJ, n, 0}; }
Role slot_r(int s, int w) { return Role{R_SLOT, s, w}; }
Role hstage_r(int k, int w) { return Role{R_HSTAGE, k, w}; }
Role hrest_r(int r, int w) { return Role{R_HREST, r, w}; }

void* rptr(ckfwi_model* m, int mode, const Role& r)
{
    const FieldGeom& f = m->fg;
    switch (r.kind) {
    case R_ZERO: return org(m->zero, f);
    case R_WORK: return org(m->work[r.idx], f);
    case R_LAM: return org(m->lam[r.idx], f);
    case R_UN: return org(m->uN, f);
    case R_TRAJ: return m->traj.as<float>() + (size_t)r.idx * f.alloc + f.origin;
    case R_HSTAGE: return org(m->hstage[r.idx][r.which], f);
    case R_HREST: return org(m->hrest[r.idx][r.which], f);
    case R_SLOT: {
        // uncompressed slots: two padded fields per slot, FP32 or 16-bit;
        // slots 1 .. host_slots in host memory, the rest in device memory
        const size_t es = mode == CKFWI_STORE_FP32 ? 4 : 2;
        const size_t fb = field_bytes(f, es), off = (size_t)f.origin * es;
        if (r.idx <= m->host_slots)
            return static_cast<char*>(m->hpool.d) + ((size_t)(r.idx - 1) * 2 + r.which) * fb + off;
        return m->pool.as<char>() + ((size_t)(r.idx - 1 - m->host_slots) * 2 + r.which) * fb + off;
    }
    default: return nullptr;
    }
}

// CKFWI_DEBUG=1 (read at the start of every gradient call): before every
// step launch the executor checks on the host that each field the step reads
// or writes lies inside the allocation its role names, and that the fields it
// writes are none of those it reads; a violation is CKFWI_EINVAL with a
// message on stderr, and nothing is launched.
bool debug_env()
{
    const char* v = std::getenv("CKFWI_DEBUG");
    return v && *v && std::strcmp(v, "0") != 0;
}

// The allocation that holds role r (base, bytes) and its element size;
// false for a role index outside its kind's range.
bool role_extent(const ckfwi_model* m, int mode, const Role& r, const char** base, size_t* bytes, size_t* es)
{
    *es = 4;
    const DevMem* d = nullptr;
    switch (r.kind) {
    case R_ZERO: d = &m->zero; break;
    case R_WORK: if (r.idx < 0 || r.idx >= 3) return false; d = &m->work[r.idx]; break;
    case R_LAM: if (r.idx < 0 || r.idx >= 3) return false; d = &m->lam[r.idx]; break;
    case R_UN: d = &m->uN; break;
    case R_TRAJ: if (r.idx < 0) return false; d = &m->traj; break;
    case R_HSTAGE: if (r.idx < 0 || r.idx >= 3 || r.which < 0 || r.which > 1) return false;
        d = &m->hstage[r.idx][r.which]; break;
    case R_HREST: if (r.idx < 0 || r.idx >= 2 || r.which < 0 || r.which > 1) return false;
        d = &m->hrest[r.idx][r.which]; break;
    case R_SLOT:
        if (r.idx < 1 || r.which < 0 || r.which > 1) return false;
        *es = mode == CKFWI_STORE_FP32 ? 4 : 2;
        if (r.idx <= m->host_slots) {
            *base = static_cast<const char*>(m->hpool.d);
            *bytes = m->hpool.bytes;
            return *base != nullptr;
        }
        d = &m->pool;
        break;
    default: return false;
    }
    *base = static_cast<const char*>(d->p);
    *bytes = d->bytes;
    return *base != nullptr;
}

// CKFWI_OK when the padded field of role r, whose element (0,0,0) is at p,
// lies inside r's allocation; else CKFWI_EINVAL and a message
int check_field(const ckfwi_model* m, int mode, const Role& r, const void* p, const char* what)
{
    const char* base = nullptr;
    size_t bytes = 0, es = 4;
    bool ok = role_extent(m, mode, r, &base, &bytes, &es);
    if (ok) {
        const char* start = static_cast<const char*>(p) - (size_t)m->fg.origin * es;
        ok = start >= base && start + field_bytes(m->fg, es) <= base + bytes;
    }
    if (!ok)
        std::fprintf(stderr, "ckfwi debug: %s (role %d, index %d, field %d) is outside its allocation\n", what,
                     r.kind, r.idx, r.which);
    return ok ? CKFWI_OK : CKFWI_EINVAL;
}

// CKFWI_EINVAL and a message when the written role w is the read role r
int check_distinct(const Role& w, const Role& r, const char* what)
{
    if (w.kind == R_NONE || w != r) return CKFWI_OK;
    std::fprintf(stderr, "ckfwi debug: %s (role %d, index %d, field %d) is both read and written\n", what, w.kind,
                 w.idx, w.which);
    return CKFWI_EINVAL;
}

struct Ctx {
    ckfwi_model* m;                 // the model (lane 0 of a batch)
    cudaStream_t st;
    long long launches = 0;
    Prof prof;
    long long count[PC_N] = {0, 0, 0, 0, 0};
    int mode = CKFWI_STORE_FP32;    // storage mode R_SLOT roles resolve for
    bool stage = false;             // FP32 host slots go through the device staging pairs
    bool pend[3] = {false, false, false};  // a copy from staging pair k to a host slot is in flight
    int sk = 0;                     // the staging pair the next host checkpoint takes
    int stage_slot[3] = {0, 0, 0};  // host slot whose checkpoint staging pair k still holds (0: none)
    int rest_slot[2] = {0, 0};      // host slot copied into restore pair r (0: none)
    int rest_fields[2] = {0, 0};    // and how many of its fields
    bool rest_pf[2] = {false, false};   // that copy is a prefetch on the copy stream (event ev_pf[r])
    int rk = 0;                     // the restore pair the next unprefetched restore takes
    bool debug = debug_env();       // host checks of every step's fields (CKFWI_DEBUG)
    // batch: every stencil step is one launch over all lanes
    std::vector<ckfwi_model*> lanes;   // empty: the model alone
    bool batch = false;
    bool issue = true;              // false: only collect the batch argument tables
    std::vector<FwdArgs> ftab;      // one row per lane and step, in launch order
    std::vector<AdjArgs> atab;
    size_t fi = 0, ai = 0;          // next row
    const FwdArgs* ftab_d = nullptr;
    const AdjArgs* atab_d = nullptr;
    const int* fstart_d = nullptr;
    const int* astart_d = nullptr;
    long long fblocks = 0, ablocks = 0;
    Tile bf{}, ba{};                // batch tile shapes; z-run length per lane in zf / za
    std::vector<int> zf, za;
    int nl() const { return lanes.empty() ? 1 : (int)lanes.size(); }
    ckfwi_model* lane(int l) const { return lanes.empty() ? m : lanes[l]; }
    void* ptr(int l, const Role& r) const { return rptr(lane(l), mode, r); }
    float* fptr(int l, const Role& r) const { return static_cast<float*>(ptr(l, r)); }
    int begin(int cls)
    {
        ++count[cls];
        if (!prof.on) return -1;
        cudaEvent_t e = prof.take();
        cudaEvent_t f = prof.take();
        if (!e || !f) return -1;
        cudaEventRecord(e, st);
        prof.marks.emplace_back(cls, (int)prof.next - 2);
        return 0;
    }
    void end(int tok)
    {
        if (tok < 0 || !prof.on) return;
        cudaEventRecord((*prof.pool)[prof.marks.back().second + 1], st);
    }
};

FwdArgs fwd_args(ckfwi_model* m)
{
    FwdArgs a{};
    a.g = m->fg;
    a.w = org(m->w, m->fg);
    a.eta = m->eta.as<float>();
    a.hdt = m->hdt;
    std::memcpy(a.c, m->c, sizeof(a.c));
    a.err = m->flags.as<int>();
    a.wait_limit = m->wait_limit;
    return a;
}

AdjArgs adj_args(ckfwi_model* m)
{
    AdjArgs a{};
    a.g = m->fg;
    a.w = org(m->w, m->fg);
    a.gacc = org(m->gacc, m->fg);
    a.eta = m->eta.as<float>();
    a.hdt = m->hdt;
    std::memcpy(a.c, m->c, sizeof(a.c));
    a.err = m->flags.as<int>();
    a.wait_limit = m->wait_limit;
    return a;
}

// receiver sampling of u^n for the model's shot
Sample sample_of(ckfwi_model* m, int n)
{
    Sample sm{};
    sm.n = m->shot.nrec;
    sm.nst = m->shot.nst;
    sm.idx = m->shot.ridx.as<long long>();
    sm.wt = m->shot.rwt.as<float>();
    sm.out = m->shot.dsim.as<float>() + (size_t)n * m->shot.nrec;
    return sm;
}

// whether a step's grid has one thread per receiver, so that it can sample
bool grid_samples(const FieldGeom& f, const Tile& t, int zlen, int nrec)
{
    const long long gx = (f.nx + t.bx - 1) / t.bx;
    const long long gy = f.dims == 3 ? (f.ny + t.by - 1) / t.by : 1;
    const long long gz = (f.nz + zlen - 1) / zlen;
    const long long tpc = (t.ver == 2 ? t.bx / 4 : (t.ver >= 3 ? t.bx / t.vec : t.bx)) * (long long)t.by;
    return gx * gy * gz * tpc >= nrec;
}

// A checkpoint slot in host memory (the second storage level).  Tensor maps
// are built on device memory only, so a step whose TMA-read operand is such
// a slot runs the register-queue kernel (bitwise the same values).
bool in_host(const ckfwi_model* m, const Role& r) { return r.kind == R_SLOT && r.idx <= m->host_slots; }
Tile host_tile(const ckfwi_model* m)
{
    Tile t = tile_at(m->fg.dims, 1, 16);
    if (!tile_supported(m->fg.dims, m->K, t)) t = tile_at(m->fg.dims, 2, 16);
    return t;
}

// OT4 steps (ot4.cu): forward, the pass computing w lap f, then the update;
// reverse, w lap of lam^j and u^{j-1}, the update, the gradient pass.  The
// reverse step j writes w lap u^{j-1} into z4[1 + j % 2] and pairs the one
// of step j + 1 with lap lam^j.
int ot4_fwd_step(ckfwi_model* m, const FwdArgs& a, const Tile& t, int ck, cudaStream_t st)
{
    const FieldGeom& f = m->fg;
    Ot4LapArgs la{};
    la.g = f;
    la.f0 = a.u;
    la.z0 = org(m->z4[0], f);
    la.w = a.w;
    std::memcpy(la.c, m->c, sizeof(la.c));
    la.smp = a.smp;
    if (t.ver == 6) CK_TRY(launch_ot4v_lap(la, t, m->K, U_FP32, st));
    else CK_TRY(launch_ot4_lap(la, t, m->K, U_FP32, st));
    Ot4FwdArgs fa{};
    fa.f = a;
    fa.f.smp = Sample{};
    fa.z = la.z0;
    std::memcpy(fa.c12, m->c12, sizeof(fa.c12));
    if (t.ver == 6) CK_TRY(launch_ot4v_fwd(fa, t, m->K, ck, st));
    else CK_TRY(launch_ot4_fwd(fa, t, m->K, ck, st));
    return CKFWI_OK;
}

int ot4_adj_step(ckfwi_model* m, const AdjArgs& a, const Tile& t, int utype, int j, cudaStream_t st)
{
    const FieldGeom& f = m->fg;
    // pass 1: Z_l, Z_u(j), and the deferred term of step j + 1
    Ot4LapArgs la{};
    la.g = f;
    la.f0 = a.l1;
    la.f1 = a.u;
    la.z0 = org(m->z4[0], f);
    la.z1 = org(m->z4[1 + (j & 1)], f);
    la.w = a.w;
    std::memcpy(la.c, m->c, sizeof(la.c));
    la.gacc = a.gacc;
    la.zu_next = j < m->g.nt ? org(m->z4[1 + ((j + 1) & 1)], f) : nullptr;
    std::memcpy(la.c12, m->c12, sizeof(la.c12));
    if (t.ver == 6) CK_TRY(launch_ot4v_lap(la, t, m->K, utype, st));
    else CK_TRY(launch_ot4_lap(la, t, m->K, utype, st));
    // pass 2: lam^{j-1} by the forward update kernel on the adjoint's fields
    Ot4FwdArgs ua{};
    ua.f.g = f;
    ua.f.u = a.l1;
    ua.f.up = a.l2;
    ua.f.w = a.w;
    ua.f.out = a.l0;
    ua.f.eta = a.eta;
    ua.f.hdt = a.hdt;
    ua.f.src = a.adj;
    ua.f.err = a.err;
    ua.z = la.z0;
    std::memcpy(ua.c12, m->c12, sizeof(ua.c12));
    if (t.ver == 6) CK_TRY(launch_ot4v_fwd(ua, t, m->K, CK_NONE, st));
    else CK_TRY(launch_ot4_fwd(ua, t, m->K, CK_NONE, st));
    // pass 3: the gradient term of lam^{j-1}
    Ot4GradArgs ga{};
    ga.g = f;
    ga.u = a.u;
    ga.zu = la.z1;
    ga.l0 = a.l0;
    ga.gacc = a.gacc;
    std::memcpy(ga.c, m->c, sizeof(ga.c));
    std::memcpy(ga.c12, m->c12, sizeof(ga.c12));
    ga.src = a.src;
    if (t.ver == 6) CK_TRY(launch_ot4v_grad(ga, t, m->K, utype, st));
    else CK_TRY(launch_ot4_grad(ga, t, m->K, utype, st));
    return CKFWI_OK;
}

// One forward step n of every lane: u -> out, optionally sampling d^n and
// writing a fused takeshot (ck, ck_u, ck_up).
// The six tensor maps of a split reverse step (launch_adjq): lam^j with the
// u box, lam^{j+1} and w with point boxes, u^{j-1} with the u box, lam^{j-1}
// and g with point boxes
int adjq_maps(ckfwi_model* m, const AdjArgs& a, CUtensorMap* mp)
{
    const int bx = tq_box_x(m->K), by = tq_box_y(m->K);
    ST_TRY(tensor_map(m, a.l1, U_FP32, bx, by, &mp[0]));
    ST_TRY(tensor_map(m, a.l2, U_FP32, 32, 16, &mp[1]));
    ST_TRY(tensor_map(m, a.w, U_FP32, 32, 16, &mp[2]));
    ST_TRY(tensor_map(m, a.u, U_FP32, bx, by, &mp[3]));
    ST_TRY(tensor_map(m, a.l0, U_FP32, 32, 16, &mp[4]));
    ST_TRY(tensor_map(m, a.gacc, U_FP32, 32, 16, &mp[5]));
    return CKFWI_OK;
}

int fwd_step(Ctx& cx, const Role& u, const Role& up, const Role& out, int n, bool record, int ck,
             const Role& ck_u, const Role& ck_up)
{
    const int NL = cx.nl();
    for (int l = 0; l < NL; ++l) {
        ckfwi_model* m = cx.lane(l);
        FwdArgs a = fwd_args(m);
        a.u = cx.fptr(l, u);
        a.up = cx.fptr(l, up);
        a.out = cx.fptr(l, out);
        a.src = m->shot.src.view;
        a.src.series = m->shot.wavelet.as<float>() + n;
        a.ck_u = cx.ptr(l, ck_u);
        a.ck_up = cx.ptr(l, ck_up);
        if (cx.debug) {
            ST_TRY(check_field(m, CKFWI_STORE_FP32, u, a.u, "forward step: u^n"));
            ST_TRY(check_field(m, CKFWI_STORE_FP32, up, a.up, "forward step: u^{n-1}"));
            ST_TRY(check_field(m, CKFWI_STORE_FP32, out, a.out, "forward step: u^{n+1}"));
            for (const Role* r : {&u, &up}) {
                ST_TRY(check_distinct(out, *r, "forward step: u^{n+1}"));
                ST_TRY(check_distinct(ck_u, *r, "forward step: checkpoint u^s"));
                ST_TRY(check_distinct(ck_up, *r, "forward step: checkpoint u^{s-1}"));
            }
            if (ck != CK_NONE) {
                const int cm = ck == CK_FP32 ? CKFWI_STORE_FP32 : CKFWI_STORE_FP16;
                if (ck != CK_FP32) ST_TRY(check_field(m, cm, ck_u, a.ck_u, "forward step: checkpoint u^s"));
                ST_TRY(check_field(m, cm, ck_up, a.ck_up, "forward step: checkpoint u^{s-1}"));
            }
        }
        const Tile& t = cx.batch ? cx.bf : m->tf;
        const int zlen = cx.batch ? cx.zf[l] : m->tf.zlen;
        bool sep = false;
        if (record) {
            const Sample sm = sample_of(m, n);
            if (grid_samples(m->fg, t, zlen, sm.n)) a.smp = sm;
            else sep = true;
            if (sep && cx.issue) {
                CK_TRY(launch_sample(a.u, sm, cx.st));
                ++cx.launches;
            }
        }
        if (cx.batch) {
            a.zlen = zlen;
            if (!cx.issue) cx.ftab.push_back(a);
            continue;
        }
        const int tok = cx.begin(PC_FWD);
        if (m->tf.ver == 8) {
            if (in_host(m, u) || in_host(m, up)) {
                // tensor maps cover device memory only: the async-copy kernel of the same tile
                Tile t4 = m->tf;
                t4.ver = 4;
                t4.pf = m->K <= 4 ? 1 : 0;
                CK_TRY(launch_fwd4(a, t4, m->K, ck, cx.st));
            } else {
                CUtensorMap tu, tp, tw;
                ST_TRY(tensor_map(m, a.u, U_FP32, tq_box_x(m->K), tq_box_y(m->K), &tu));
                ST_TRY(tensor_map(m, a.up, U_FP32, 32, 16, &tp));
                ST_TRY(tensor_map(m, a.w, U_FP32, 32, 16, &tw));
                CK_TRY(launch_fwdq(a, tu, tp, tw, m->tf, m->K, ck, cx.st));
            }
        } else if (m->tf.ver == 7) {
            CK_TRY(launch_fwd5(a, m->tf, m->K, ck, cx.st));
        } else if (m->tf.ver >= 5) {
            ST_TRY(ot4_fwd_step(m, a, m->tf, ck, cx.st));
            ++cx.launches;
        } else if (m->tf.ver == 2 && in_host(m, u)) {
            CK_TRY(launch_fwd(a, host_tile(m), m->K, ck, cx.st));
        } else if (m->tf.ver == 4) {
            CK_TRY(launch_fwd4(a, m->tf, m->K, ck, cx.st));
        } else if (m->tf.ver == 3) {
            CK_TRY(launch_fwd3(a, m->tf, m->K, ck, cx.st));
        } else if (m->tf.ver == 2) {
            CUtensorMap tm;
            ST_TRY(tensor_map(m, a.u, U_FP32, tma_tile_x() + 2 * tma_halo_x(m->K), m->tf.by + 2 * m->K, &tm));
            CK_TRY(launch_fwd_tma(a, tm, m->tf, m->K, ck, cx.st));
        } else {
            CK_TRY(launch_fwd(a, m->tf, m->K, ck, cx.st));
        }
        cx.end(tok);
        ++cx.launches;
    }
    if (cx.batch) {
        if (cx.issue) {
            const int tok = cx.begin(PC_FWD);
            BatchLaunch<FwdArgs> b{cx.ftab_d + cx.fi, cx.fstart_d, NL, cx.m->fg.dims, cx.fblocks};
            if (cx.bf.ver == 7) CK_TRY(launch_fwd5_batch(b, cx.bf, cx.m->K, ck, cx.st));
            else if (cx.bf.ver == 4) CK_TRY(launch_fwd4_batch(b, cx.bf, cx.m->K, ck, cx.st));
            else if (cx.bf.ver == 3) CK_TRY(launch_fwd3_batch(b, cx.bf, cx.m->K, ck, cx.st));
            else CK_TRY(launch_fwd_batch(b, cx.bf, cx.m->K, ck, cx.st));
            cx.end(tok);
            ++cx.launches;
        }
        cx.fi += NL;
    }
    return CKFWI_OK;
}

// One fused reverse step j of every lane: lam^{j-1} from lam^j, lam^{j+1}
// and the residual row j; gacc += lam^{j-1} (lap u^{j-1} + source^{j-1}).
int adj_step(Ctx& cx, const Role& l1, const Role& l2, const Role& l0, const Role& u, int utype, int j)
{
    const int NL = cx.nl();
    for (int l = 0; l < NL; ++l) {
        ckfwi_model* m = cx.lane(l);
        AdjArgs a = adj_args(m);
        a.l1 = cx.fptr(l, l1);
        a.l2 = cx.fptr(l, l2);
        a.l0 = cx.fptr(l, l0);
        a.u = cx.ptr(l, u);
        if (cx.debug) {
            ST_TRY(check_field(m, CKFWI_STORE_FP32, l1, a.l1, "reverse step: lambda^j"));
            ST_TRY(check_field(m, CKFWI_STORE_FP32, l2, a.l2, "reverse step: lambda^{j+1}"));
            ST_TRY(check_field(m, CKFWI_STORE_FP32, l0, a.l0, "reverse step: lambda^{j-1}"));
            ST_TRY(check_field(m, utype == U_FP32 ? CKFWI_STORE_FP32 : CKFWI_STORE_FP16, u, a.u,
                               "reverse step: u^{j-1}"));
            ST_TRY(check_distinct(l0, l1, "reverse step: lambda^{j-1}"));
            ST_TRY(check_distinct(l0, l2, "reverse step: lambda^{j-1}"));
        }
        a.adj = m->shot.adj.view;
        a.adj.series = m->shot.resid.as<float>() + (size_t)j * m->shot.nrec;
        a.src = m->shot.src.view;
        a.src.series = m->shot.wavelet.as<float>() + (j - 1);
        if (cx.batch) {
            a.zlen = cx.za[l];
            if (!cx.issue) cx.atab.push_back(a);
            continue;
        }
        const int tok = cx.begin(PC_ADJ);
        if (m->ta.ver == 8 && (utype != U_FP32 || in_host(m, u))) {
            // tensor maps cover FP32 device fields only: the lean kernel of the same tile
            Tile t7 = m->ta;
            t7.ver = 7;
            t7.pf = 1;
            CK_TRY(launch_adj5(a, t7, m->K, utype, cx.st));
        } else if (m->ta.ver == 8) {
            CUtensorMap mp[6];
            ST_TRY(adjq_maps(m, a, mp));
            CK_TRY(launch_adjq(a, mp, m->ta, m->K, cx.st));
            ++cx.launches;
        } else if (m->ta.ver == 7) {
            CK_TRY(launch_adj5(a, m->ta, m->K, utype, cx.st));
        } else if (m->ta.ver >= 5) {
            ST_TRY(ot4_adj_step(m, a, m->ta, utype, j, cx.st));
            cx.launches += 2;
        } else if (m->ta.ver == 2 && in_host(m, u)) {
            CK_TRY(launch_adj(a, host_tile(m), m->K, utype, cx.st));
        } else if (m->ta.ver == 4) {
            CK_TRY(launch_adj4(a, m->ta, m->K, utype, cx.st));
        } else if (m->ta.ver == 3) {
            CK_TRY(launch_adj3(a, m->ta, m->K, utype, cx.st));
        } else if (m->ta.ver == 2) {
            CUtensorMap tl, tu;
            const int bx = tma_tile_x() + 2 * tma_halo_x(m->K), by = m->ta.by + 2 * m->K;
            ST_TRY(tensor_map(m, a.l1, U_FP32, bx, by, &tl));
            ST_TRY(tensor_map(m, a.u, utype, bx, by, &tu));
            CK_TRY(launch_adj_tma(a, tl, tu, m->ta, m->K, utype, cx.st));
        } else {
            CK_TRY(launch_adj(a, m->ta, m->K, utype, cx.st));
        }
        cx.end(tok);
        ++cx.launches;
    }
    if (cx.batch) {
        if (cx.issue) {
            const int tok = cx.begin(PC_ADJ);
            BatchLaunch<AdjArgs> b{cx.atab_d + cx.ai, cx.astart_d, NL, cx.m->fg.dims, cx.ablocks};
            if (cx.ba.ver == 7) CK_TRY(launch_adj5_batch(b, cx.ba, cx.m->K, utype, cx.st));
            else if (cx.ba.ver == 3) CK_TRY(launch_adj3_batch(b, cx.ba, cx.m->K, utype, cx.st));
            else CK_TRY(launch_adj_batch(b, cx.ba, cx.m->K, utype, cx.st));
            cx.end(tok);
            ++cx.launches;
        }
        cx.ai += NL;
    }
    return CKFWI_OK;
}

// d^N = P u^N of every lane
int sample_last(Ctx& cx, const Role& uN)
{
    if (!cx.issue) return CKFWI_OK;
    for (int l = 0; l < cx.nl(); ++l) {
        ckfwi_model* m = cx.lane(l);
        CK_TRY(launch_sample(cx.fptr(l, uN), sample_of(m, m->g.nt), cx.st));
        ++cx.launches;
    }
    return CKFWI_OK;
}

// max |u^N| of every lane (the wavefield's scale, reported beside a codec
// tolerance); the second word of the lane's phi buffer, zeroed at the start
// of the gradient
int field_absmax(Ctx& cx, const Role& uN)
{
    if (!cx.issue) return CKFWI_OK;
    for (int l = 0; l < cx.nl(); ++l) {
        ckfwi_model* m = cx.lane(l);
        CK_TRY(launch_absmax(cx.fptr(l, uN), m->fg, reinterpret_cast<unsigned*>(m->phi.as<double>() + 1), cx.st));
        ++cx.launches;
    }
    return CKFWI_OK;
}

// residual r = d - d_obs and the FP64 misfit of every lane
int residual(Ctx& cx)
{
    if (!cx.issue) return CKFWI_OK;
    for (int l = 0; l < cx.nl(); ++l) {
        ckfwi_model* m = cx.lane(l);
        CK_TRY(launch_residual(m->shot.dsim.as<float>(), m->shot.dobs.as<float>(), m->shot.resid.as<float>(),
                               m->g.nt + 1, m->shot.nrec, m->partials.as<double>(), m->nparts,
                               m->phi.as<double>(), cx.st));
        cx.launches += 2;
    }
    return CKFWI_OK;
}

int tensor_map(ckfwi_model* m, const void* origin_ptr, int utype, int bx, int by, CUtensorMap* out)
{
    const FieldGeom& f = m->fg;
    const int es = utype == U_FP32 ? 4 : 2;
    const void* base = static_cast<const char*>(origin_ptr) - f.origin * es;
    const auto key = std::make_tuple(base, utype, bx, by);
    auto it = m->tmaps.find(key);
    if (it != m->tmaps.end()) {
        *out = it->second;
        return CKFWI_OK;
    }
    EncodeTiled enc = encode_fn();
    if (!enc || f.dims != 3) return CKFWI_ECUDA;
    const cuuint64_t py = (cuuint64_t)f.ny + 2 * f.H, pz = (cuuint64_t)f.nz + 2 * f.H;
    const cuuint64_t dims[3] = {(cuuint64_t)f.px, py, pz};
    const cuuint64_t strides[2] = {(cuuint64_t)f.px * es, (cuuint64_t)f.pxy * es};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = utype == U_FP32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : utype == U_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                     : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    CUtensorMap tm;
    if (enc(&tm, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return CKFWI_ECUDA;
    m->tmaps.emplace(key, tm);
    *out = tm;
    return CKFWI_OK;
}

// --------------------------------------------------------------- autotune
int autotune(ckfwi_model* m, cudaStream_t st)
{
    if (m->tuned) return CKFWI_OK;
    const FieldGeom& f = m->fg;
    // candidate z-run lengths: whole columns, and runs giving >= 4 CTAs per SM
    int dev = 0;
    cudaGetDevice(&dev);
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    std::vector<Tile> cands;
    // Candidate z-run lengths for a tile with `cols` column blocks: runs
    // giving about 2-16 CTAs per SM, and every run length from 4 to 32
    // planes, among which are the ones whose CTA count fills the last wave
    // of resident CTAs (a grid of 2.1 waves runs as 3).  The timings pick.
    auto zlens = [&](long long cols) {
        std::vector<int> zl;
        auto add = [&](int z) {
            z = std::max(4, std::min(z, f.nz));
            if (std::find(zl.begin(), zl.end(), z) == zl.end()) zl.push_back(z);
        };
        for (int target : {2, 4, 8, 16}) {
            long long nzc = (target * (long long)nsm + cols - 1) / cols;
            nzc = std::max<long long>(1, std::min<long long>(nzc, f.nz));
            add((int)((f.nz + nzc - 1) / nzc));
        }
        for (int z = 4; z <= 32; ++z) add(z);
        return zl;
    };
    // the OT4 kernel has its own two-pass kernels, tried alone
    for (int i = 0; m->ot == 4 && i < ot4_shape_count(f.dims); ++i) {
        const Tile t0 = ot4_tile_at(f.dims, i, f.nz);
        if (!ot4_supported(f.dims, m->K, t0)) continue;
        const long long cols = (long long)((f.nx + t0.bx - 1) / t0.bx) * (f.dims == 3 ? (f.ny + t0.by - 1) / t0.by : 1);
        for (int z : zlens(cols)) cands.push_back(ot4_tile_at(f.dims, i, z));
    }
    if (m->ot == 4 && f.dims == 3 && v3_fits(f, m->K)) {
        for (int vec : {4, 2}) {
            Tile t0;
            t0.ver = 6;
            t0.bx = 32;
            t0.by = 16;
            t0.vec = vec;
            t0.zlen = f.nz;
            if (!ot4v_supported(f.dims, m->K, t0, false)) continue;
            const long long cols = (long long)((f.nx + 31) / 32) * ((f.ny + 15) / 16);
            for (int z : zlens(cols)) {
                t0.zlen = z;
                cands.push_back(t0);
            }
        }
    }
    for (int i = 0; m->ot == 2 && i < tile_count(f.dims); ++i) {
        Tile t0 = tile_at(f.dims, i, f.nz);
        if (!tile_supported(f.dims, m->K, t0)) continue;
        const long long cols = (long long)((f.nx + t0.bx - 1) / t0.bx) * (f.dims == 3 ? (f.ny + t0.by - 1) / t0.by : 1);
        for (int z : zlens(cols)) cands.push_back(tile_at(f.dims, i, z));
    }
    // vector-blocked kernels (3D)
    if (m->ot == 2 && f.dims == 3 && v3_fits(f, m->K)) {
        for (int i = 0; i < v3_shape_count(); ++i) {
            const Tile t0 = v3_tile_at(i, f.nz);
            if (!v3_supported(f.dims, m->K, t0)) continue;
            const long long cols = (long long)((f.nx + t0.bx - 1) / t0.bx) * ((f.ny + t0.by - 1) / t0.by);
            for (int z : zlens(cols)) {
                cands.push_back(v3_tile_at(i, z));
                Tile t4 = v3_tile_at(i, z);     // the same shape fed by asynchronous copies
                t4.ver = 4;
                if (v4_supported(f.dims, m->K, t4)) cands.push_back(t4);
                t4.pf = 1;                       // one plane of prefetch, six CTAs per SM
                if (v4_supported(f.dims, m->K, t4)) cands.push_back(t4);
                Tile t7 = v3_tile_at(i, z);     // the lean generation, one or two planes per step
                t7.ver = 7;
                for (int np : {1, 2}) {
                    t7.pf = np;
                    if (v5_supported(f.dims, m->K, t7)) cands.push_back(t7);
                }
                Tile t8 = v3_tile_at(i, z);     // the forward step fed by tensor copies
                t8.ver = 8;
                for (int pf : {1, 2}) {
                    t8.pf = pf;
                    if (encode_fn() && tq_supported(f.dims, m->K, t8)) cands.push_back(t8);
                }
            }
        }
    }
    const bool tma_ok = encode_fn() != nullptr;
    // TMA kernels run a persistent grid; their zlen field is the CTAs per SM
    for (int ty : {8, 16}) {
        if (m->ot != 2 || !tma_ok || !tma_supported(f.dims, m->K, ty)) continue;
        for (int per_sm : {1, 2, 3}) {
            Tile t;
            t.bx = 64;
            t.by = ty;
            t.zlen = per_sm;
            t.ver = 2;
            cands.push_back(t);
        }
    }
    // time the forward and the reverse kernel on the model's own buffers
    cudaEvent_t e0, e1;
    CK_TRY(cudaEventCreate(&e0));
    CK_TRY(cudaEventCreate(&e1));
    FwdArgs a = fwd_args(m);
    a.u = org(m->work[0], f);
    a.up = org(m->work[1], f);
    a.out = org(m->work[2], f);
    AdjArgs b{};
    b.g = f;
    b.l1 = org(m->lam[0], f);
    b.l2 = org(m->lam[1], f);
    b.l0 = org(m->lam[2], f);
    b.u = org(m->work[0], f);
    b.w = org(m->w, f);
    b.gacc = org(m->gacc, f);
    b.eta = m->eta.as<float>();
    b.hdt = m->hdt;
    std::memcpy(b.c, m->c, sizeof(b.c));
    b.err = m->flags.as<int>();
    b.wait_limit = m->wait_limit;
    const int reps = 3;
    CUtensorMap tm_u, tm_l;
    auto go = [&](const Tile& t, int pass) -> int {
        if (t.ver == 8 && pass == 1) {
            CUtensorMap mp[6];
            ST_TRY(adjq_maps(m, b, mp));
            CK_TRY(launch_adjq(b, mp, t, m->K, st));
        } else if (t.ver == 8) {
            CUtensorMap tu, tp, tw;
            ST_TRY(tensor_map(m, a.u, U_FP32, tq_box_x(m->K), tq_box_y(m->K), &tu));
            ST_TRY(tensor_map(m, a.up, U_FP32, 32, 16, &tp));
            ST_TRY(tensor_map(m, a.w, U_FP32, 32, 16, &tw));
            CK_TRY(launch_fwdq(a, tu, tp, tw, t, m->K, CK_NONE, st));
        } else if (t.ver == 7) {
            if (pass == 0) CK_TRY(launch_fwd5(a, t, m->K, CK_NONE, st));
            else CK_TRY(launch_adj5(b, t, m->K, U_FP32, st));
        } else if (t.ver >= 5) {
            if (pass == 0) ST_TRY(ot4_fwd_step(m, a, t, CK_NONE, st));
            else ST_TRY(ot4_adj_step(m, b, t, U_FP32, m->g.nt, st));
        } else if (t.ver == 4) {
            if (pass == 0) CK_TRY(launch_fwd4(a, t, m->K, CK_NONE, st));
            else CK_TRY(launch_adj4(b, t, m->K, U_FP32, st));
        } else if (t.ver == 3) {
            if (pass == 0) CK_TRY(launch_fwd3(a, t, m->K, CK_NONE, st));
            else CK_TRY(launch_adj3(b, t, m->K, U_FP32, st));
        } else if (t.ver == 2) {
            const int bx = tma_tile_x() + 2 * tma_halo_x(m->K), by = t.by + 2 * m->K;
            ST_TRY(tensor_map(m, a.u, U_FP32, bx, by, &tm_u));
            ST_TRY(tensor_map(m, b.l1, U_FP32, bx, by, &tm_l));
            if (pass == 0) CK_TRY(launch_fwd_tma(a, tm_u, t, m->K, CK_NONE, st));
            else CK_TRY(launch_adj_tma(b, tm_l, tm_u, t, m->K, U_FP32, st));
        } else {
            if (pass == 0) CK_TRY(launch_fwd(a, t, m->K, CK_NONE, st));
            else CK_TRY(launch_adj(b, t, m->K, U_FP32, st));
        }
        return CKFWI_OK;
    };
    // a forced tile (CKFWI_TILE_FWD / CKFWI_TILE_ADJ = "ver,bx,by,zlen[,vec]") skips the search
    auto forced = [&](const char* name, Tile* t, bool reverse) {
        const char* v = std::getenv(name);
        if (!v) return false;
        Tile u;
        const int nf = std::sscanf(v, "%d,%d,%d,%d,%d,%d", &u.ver, &u.bx, &u.by, &u.zlen, &u.vec, &u.pf);
        if (nf < 4 || u.zlen < 1) return false;
        if (nf < 5) u.vec = 1;
        if (nf < 6) u.pf = 0;
        if ((u.ver == 5 || u.ver == 6) != (m->ot == 4)) return false;
        const bool okv = u.ver == 8   ? tma_ok && tq_supported(f.dims, m->K, u) && v3_fits(f, m->K)
                         : u.ver == 7 ? v5_supported(f.dims, m->K, u) && v3_fits(f, m->K)
                         : u.ver == 6 ? ot4v_supported(f.dims, m->K, u, reverse) && v3_fits(f, m->K)
                         : u.ver == 5 ? ot4_supported(f.dims, m->K, u)
                         : u.ver == 4 ? v4_supported(f.dims, m->K, u) && v3_fits(f, m->K)
                         : u.ver == 3 ? v3_supported(f.dims, m->K, u) && v3_fits(f, m->K)
                         : u.ver == 2 ? (tma_ok && u.bx == 64 && tma_supported(f.dims, m->K, u.by))
                                      : tile_supported(f.dims, m->K, u);
        if (!okv) return false;
        *t = u;
        return true;
    };
    const bool ff = forced("CKFWI_TILE_FWD", &m->tf, false), fa = forced("CKFWI_TILE_ADJ", &m->ta, true);
    const bool verbose = std::getenv("CKFWI_VERBOSE") != nullptr;
    // time one candidate: the median of `rounds` timings of `reps` launches
    auto time_of = [&](const Tile& t, int pass, int rounds, float* out) -> int {
        std::vector<float> v;
        for (int r = 0; r < rounds; ++r) {
            CK_TRY(cudaEventRecord(e0, st));
            for (int k = 0; k < reps; ++k) ST_TRY(go(t, pass));
            CK_TRY(cudaEventRecord(e1, st));
            CK_TRY(cudaEventSynchronize(e1));
            float ms = 0;
            CK_TRY(cudaEventElapsedTime(&ms, e0, e1));
            v.push_back(ms / reps);
        }
        std::sort(v.begin(), v.end());
        *out = v[v.size() / 2];
        return CKFWI_OK;
    };
    // bring the clocks up before anything is timed
    if (!cands.empty()) {
        for (int k = 0; k < 30; ++k) ST_TRY(go(cands[0], k & 1));
        CK_TRY(cudaStreamSynchronize(st));
    }
    for (int pass = 0; pass < 2; ++pass) {
        if ((pass == 0 && ff) || (pass == 1 && fa)) continue;
        // a first pass over every candidate, then the best four again with
        // more rounds (single timings of ~100 us launches vary by several %)
        std::vector<std::pair<float, size_t>> t1;
        for (size_t i = 0; i < cands.size(); ++i) {
            // vector-blocked OT4 reverse steps come in one vector width only
            if (cands[i].ver == 6 && !ot4v_supported(f.dims, m->K, cands[i], pass == 1)) continue;
            ST_TRY(go(cands[i], pass));
            float ms = 0;
            ST_TRY(time_of(cands[i], pass, 3, &ms));
            t1.emplace_back(ms, i);
            if (verbose)
                std::fprintf(stderr, "ckfwi autotune %s ver %d tile %dx%d vec %d zlen %d: %.1f us\n",
                             pass ? "adj" : "fwd", cands[i].ver, cands[i].bx, cands[i].by, cands[i].vec,
                             cands[i].zlen, 1000.0f * ms);
        }
        std::sort(t1.begin(), t1.end());
        float best = 1e30f;
        for (size_t k = 0; k < t1.size() && k < 4; ++k) {
            const Tile& t = cands[t1[k].second];
            float ms = 0;
            ST_TRY(time_of(t, pass, 7, &ms));
            if (verbose)
                std::fprintf(stderr, "ckfwi autotune %s final ver %d tile %dx%d vec %d zlen %d pf %d: %.1f us\n",
                             pass ? "adj" : "fwd", t.ver, t.bx, t.by, t.vec, t.zlen, t.pf, 1000.0f * ms);
            if (ms < best) {
                best = ms;
                (pass == 0 ? m->tf : m->ta) = t;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the probe runs wrote into working buffers; clear them
    for (int i = 0; i < 3; ++i) {
        CK_TRY(cudaMemsetAsync(m->work[i].p, 0, m->work[i].bytes, st));
        CK_TRY(cudaMemsetAsync(m->lam[i].p, 0, m->lam[i].bytes, st));
    }
    CK_TRY(cudaMemsetAsync(m->gacc.p, 0, m->gacc.bytes, st));
    for (int i = 0; i < 3; ++i)
        if (m->z4[i].p) CK_TRY(cudaMemsetAsync(m->z4[i].p, 0, m->z4[i].bytes, st));
    CK_TRY(cudaStreamSynchronize(st));
    m->tuned = true;
    return CKFWI_OK;
}

int reset_flags(ckfwi_model* m, cudaStream_t st)
{
    CK_TRY(cudaMemsetAsync(m->flags.p, 0, m->flags.bytes, st));
    return CKFWI_OK;
}

int read_flags(ckfwi_model* m, cudaStream_t st, int* fl)
{
    int h[4] = {0, 0, 0, 0};
    CK_TRY(cudaMemcpyAsync(h, m->flags.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK_TRY(cudaStreamSynchronize(st));
    // flags[0]: FP16 overflow (1); flags[1]: codec bits (1 nonfinite, 2 overflow, 4 corrupt)
    *fl = 0;
    if (h[1] & 2) *fl = CKFWI_POOL_OVERFLOW;
    else if (h[1] & 4) *fl = CKFWI_CORRUPT;
    else if (h[0] & 8) *fl = CKFWI_TIMEOUT;
    else if ((h[0] & 1) || (h[1] & 1)) *fl = CKFWI_NONFINITE;
    return CKFWI_OK;
}

// ------------------------------------------------------------ gradient run
struct State {
    Role cur, prev;
    int tcur, tprev;    // U_FP32 / U_BF16 / U_FP16
};

// the state reads device pair idx of this kind (a staging or a restore pair)
bool reads_pair(const State& st, int kind, int idx)
{
    return (st.cur.kind == kind && st.cur.idx == idx) || (st.prev.kind == kind && st.prev.idx == idx);
}

struct RunCfg {
    int N, M, mode;
    float tol_f;          // CODEC: the bound; CODEC_RATE: the rate (a graph key)
    bool store_all;
    bool codec;           // CODEC or CODEC_RATE: checkpoints in the stream pool
    int rate;             // CODEC_RATE: bits per value
};

CodecView field_view(const FieldGeom& f)
{
    CodecView v{};
    v.dims = f.dims;
    v.nz = f.nz;
    v.ny = f.ny;
    v.nx = f.nx;
    v.py = f.px;
    v.pz = f.pxy;
    v.aligned = true;
    return v;
}

// a working field that holds neither the current nor the previous state
Role pick_free(const State& s)
{
    for (int i = 0; i < 3; ++i)
        if (work_r(i) != s.cur && work_r(i) != s.prev) return work_r(i);
    return NONE_R;
}

// An NVTX range for the lifetime of the object (a no-op without a tool
// attached), with an integer payload
struct NvtxRange {
    NvtxRange(const char* name, long long payload)
    {
        nvtxEventAttributes_t a{};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        a.payloadType = NVTX_PAYLOAD_TYPE_INT64;
        a.payload.llValue = payload;
        nvtxRangePushEx(&a);
    }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
const char* const kActionRange[4] = {"ckfwi advance", "ckfwi takeshot", "ckfwi restore", "ckfwi youturn"};

// The recorded part of a gradient: everything between "inputs staged" and
// "outputs ready" (this is what a CUDA graph captures).  Runs every lane of
// the context through the same schedule.
int run_body(Ctx& cx, const RunCfg& rc, const std::vector<Action>& acts, long long* counters)
{
    NvtxRange whole("ckfwi gradient", (long long)cx.nl());
    const int NL = cx.nl();
    const int N = rc.N;
    if (cx.issue) {
        for (int l = 0; l < NL; ++l) {
            ckfwi_model* m = cx.lane(l);
            for (int i = 0; i < 3; ++i) CK_TRY(cudaMemsetAsync(m->lam[i].p, 0, m->lam[i].bytes, cx.st));
            CK_TRY(cudaMemsetAsync(m->gacc.p, 0, m->gacc.bytes, cx.st));
            CK_TRY(cudaMemsetAsync(m->shot.dsim.p, 0, m->shot.dsim.bytes, cx.st));
            CK_TRY(cudaMemsetAsync(m->phi.as<double>() + 1, 0, sizeof(double), cx.st));
        }
    }
    int li = 0;   // lam rotation: lam[li] = lam^{j}, lam[(li+1)%3] = lam^{j+1}
    auto reverse = [&](int s, const Role& u, int ut) -> int {
        ST_TRY(adj_step(cx, lam_r(li), lam_r((li + 1) % 3), lam_r((li + 2) % 3), u, ut, s + 1));
        li = (li + 2) % 3;   // new lam^{j} = old lam^{j-1}, lam^{j+1} = old lam^{j}
        return CKFWI_OK;
    };
    long long fsteps = 0;
    if (rc.store_all) {
        {
            NvtxRange range(kActionRange[ACT_ADVANCE], 0);
            for (int n = 0; n < N; ++n) {
                const Role u = n == 0 ? ZERO_R : traj_r(n);
                const Role up = n <= 1 ? ZERO_R : traj_r(n - 1);
                const Role out = (n + 1 < N) ? traj_r(n + 1) : UN_R;
                ST_TRY(fwd_step(cx, u, up, out, n, true, CK_NONE, NONE_R, NONE_R));
                ++fsteps;
            }
            ST_TRY(sample_last(cx, UN_R));
            ST_TRY(field_absmax(cx, UN_R));
            ST_TRY(residual(cx));
        }
        NvtxRange range(kActionRange[ACT_YOUTURN], N - 1);
        for (int s = N - 1; s >= 0; --s) ST_TRY(reverse(s, s == 0 ? ZERO_R : traj_r(s), U_FP32));
        counters[0] = fsteps;
        return CKFWI_OK;
    }
    // Revolve
    const int ut_slot = rc.mode == CKFWI_STORE_BF16 ? U_BF16 : (rc.mode == CKFWI_STORE_FP16 ? U_FP16 : U_FP32);
    // codec: slotbase[0..M] are the slots' start words, [M+1..2M] the
    // start words of their second field
    auto sbase = [&](ckfwi_model* m, int slot) { return m->slotbase.as<long long>() + slot; };
    auto smid = [&](ckfwi_model* m, int slot) { return m->slotbase.as<long long>() + (rc.M + 1) + slot; };
    if (rc.codec && cx.issue) {
        for (int l = 0; l < NL; ++l) {
            ckfwi_model* m = cx.lane(l);
            CK_TRY(cudaMemsetAsync(m->slotbase.p, 0, sizeof(long long) * 2, cx.st));
            CK_TRY(cudaMemsetAsync(m->statw.p, 0, m->statw.bytes, cx.st));
        }
    }
    long long ncomp = 0;   // compressions per lane

    State st{ZERO_R, ZERO_R, U_FP32, U_FP32};
    bool first_sweep = true;
    for (size_t ai = 0; ai < acts.size(); ++ai) {
        const Action& A = acts[ai];
        NvtxRange range(kActionRange[A.op & 3], A.a);
        const bool next_take = ai + 1 < acts.size() && acts[ai + 1].op == ACT_TAKESHOT;
        const bool next_turn = ai + 1 < acts.size() && acts[ai + 1].op == ACT_YOUTURN;
        if (A.op == ACT_ADVANCE) {
            for (int i = 0; i < A.b; ++i) {
                const int n = A.a + i;
                const bool last = i == A.b - 1;
                int ck = CK_NONE;
                Role cku = NONE_R, ckup = NONE_R;
                Role out = pick_free(st);
                int staged = -1;             // staging pair of a host-slot checkpoint
                if (last && next_take && !rc.codec) {
                    const int slot = acts[ai + 1].b;
                    if (rc.mode == CKFWI_STORE_FP32 && cx.stage && slot <= cx.m->host_slots) {
                        // into a device staging pair (not one the step reads), copied to the host slot below
                        staged = cx.sk;
                        for (int t = 0; t < 3 && reads_pair(st, R_HSTAGE, staged); ++t) staged = (staged + 1) % 3;
                        cx.sk = (staged + 1) % 3;
                        if (cx.pend[staged]) CK_TRY(cudaStreamWaitEvent(cx.st, cx.m->ev_done[staged], 0));
                        cx.pend[staged] = false;
                        // the slot's older copies on the device are stale from here on
                        for (int k = 0; k < 3; ++k)
                            if (cx.stage_slot[k] == slot) cx.stage_slot[k] = 0;
                        for (int r = 0; r < 2; ++r)
                            if (cx.rest_slot[r] == slot) cx.rest_slot[r] = 0;
                        cx.stage_slot[staged] = slot;
                        out = hstage_r(staged, 0);
                        ck = CK_FP32;
                        ckup = hstage_r(staged, 1);
                    } else if (rc.mode == CKFWI_STORE_FP32) {
                        out = slot_r(slot, 0);   // u^{n+1} straight into the slot
                        ck = CK_FP32;
                        ckup = slot_r(slot, 1);
                    } else {
                        ck = rc.mode == CKFWI_STORE_BF16 ? CK_BF16 : CK_FP16;
                        cku = slot_r(slot, 0);
                        ckup = slot_r(slot, 1);
                    }
                }
                ST_TRY(fwd_step(cx, st.cur, st.prev, out, n, first_sweep, ck, cku, ckup));
                ++fsteps;
                if (staged >= 0) {
                    // the pair to its host slot on the copy stream, overlapped with the next steps
                    ckfwi_model* m = cx.m;
                    const size_t fb = field_bytes(m->fg);
                    char* hs = static_cast<char*>(m->hpool.p) + (size_t)(acts[ai + 1].b - 1) * 2 * fb;
                    CK_TRY(cudaEventRecord(m->ev_fork, cx.st));
                    CK_TRY(cudaStreamWaitEvent(m->side, m->ev_fork, 0));
                    for (int w = 0; w < 2; ++w)
                        CK_TRY(cudaMemcpyAsync(hs + w * fb, m->hstage[staged][w].p, fb, cudaMemcpyDefault, m->side));
                    CK_TRY(cudaEventRecord(m->ev_done[staged], m->side));
                    cx.pend[staged] = true;
                }
                st.prev = st.cur;
                st.tprev = st.tcur;
                st.cur = out;
                st.tcur = U_FP32;
            }
        } else if (A.op == ACT_TAKESHOT) {
            if (rc.codec) {
                if (cx.issue) {
                    // a field into the pool at *from, its end written to *to
                    auto comp = [&](ckfwi_model* m, const float* x, const long long* from, long long* to,
                                    unsigned long long* sw) -> cudaError_t {
                        if (rc.rate)
                            return codec_rate_compress_dev(x, field_view(m->fg), rc.rate, m->pool.as<uint32_t>(), from,
                                                           m->cap_words, to, m->flags.as<int>() + 1, sw, cx.st);
                        return codec_compress_dev(x, field_view(m->fg), rc.tol_f, m->pool.as<uint32_t>(), from,
                                                  m->cap_words, to, m->scratch.p, m->flags.as<int>() + 1, sw, cx.st);
                    };
                    int tok = cx.begin(PC_COMP);
                    for (int l = 0; l < NL; ++l) {
                        ckfwi_model* m = cx.lane(l);
                        unsigned long long* sw = m->statw.as<unsigned long long>();
                        CK_TRY(comp(m, cx.fptr(l, st.cur), sbase(m, A.b), smid(m, A.b), sw + ncomp));
                    }
                    cx.end(tok);
                    tok = cx.begin(PC_COMP);
                    for (int l = 0; l < NL; ++l) {
                        ckfwi_model* m = cx.lane(l);
                        unsigned long long* sw = m->statw.as<unsigned long long>();
                        CK_TRY(comp(m, cx.fptr(l, st.prev), smid(m, A.b), sbase(m, A.b + 1), sw + ncomp + 1));
                    }
                    cx.end(tok);
                    cx.launches += 4LL * NL;   // two launches per field in either mode
                }
                ncomp += 2;
            }
        } else if (A.op == ACT_RESTORE) {
            if (A.b == 0) {
                st = State{ZERO_R, ZERO_R, U_FP32, U_FP32};
            } else if (rc.mode == CKFWI_STORE_FP32 && cx.stage && A.b <= cx.m->host_slots) {
                // a host slot: from the staging pair that still holds its
                // checkpoint, from a restore pair it was copied into, or
                // copied now
                ckfwi_model* m = cx.m;
                const size_t fb = field_bytes(m->fg);
                const int need = next_turn ? 1 : 2;   // a reverse step needs u^s only
                int k = -1, r = -1;
                for (int q = 0; q < 3; ++q)
                    if (cx.stage_slot[q] == A.b) k = q;
                for (int q = 0; q < 2 && k < 0; ++q)
                    if (cx.rest_slot[q] == A.b && cx.rest_fields[q] >= need) r = q;
                if (k >= 0) {
                    st = State{hstage_r(k, 0), hstage_r(k, 1), U_FP32, U_FP32};
                } else {
                    if (r >= 0) {
                        if (cx.rest_pf[r]) CK_TRY(cudaStreamWaitEvent(cx.st, m->ev_pf[r], 0));
                    } else {
                        // a pair with no prefetch in flight, else the next in turn
                        r = !cx.rest_pf[cx.rk] ? cx.rk : (!cx.rest_pf[cx.rk ^ 1] ? cx.rk ^ 1 : cx.rk);
                        cx.rk = r ^ 1;
                        if (cx.rest_pf[r]) CK_TRY(cudaStreamWaitEvent(cx.st, m->ev_pf[r], 0));
                        // copies to the host still in flight (none of this slot's: it would be staged)
                        for (int q = 0; q < 3; ++q)
                            if (cx.pend[q]) CK_TRY(cudaStreamWaitEvent(cx.st, m->ev_done[q], 0));
                        const char* hs = static_cast<const char*>(m->hpool.p) + (size_t)(A.b - 1) * 2 * fb;
                        for (int w = 0; w < need; ++w)
                            CK_TRY(cudaMemcpyAsync(m->hrest[r][w].p, hs + w * fb, fb, cudaMemcpyDefault, cx.st));
                        cx.rest_slot[r] = A.b;
                        cx.rest_fields[r] = need;
                    }
                    cx.rest_pf[r] = false;
                    st = State{hrest_r(r, 0), hrest_r(r, 1), U_FP32, U_FP32};
                }
                // Prefetch the next host restore whose slot no device pair
                // holds and that no checkpoint rewrites first, into a restore
                // pair the state does not use, unless that pair's slot is
                // restored before it.
                int o = -1;
                if (!reads_pair(st, R_HREST, 0)) o = 0;
                if (!reads_pair(st, R_HREST, 1) && (o < 0 || cx.rest_slot[o] != 0)) o = 1;
                std::vector<int> taken;
                for (size_t aj = ai + 1; o >= 0 && aj < acts.size(); ++aj) {
                    const Action& B = acts[aj];
                    if (B.op == ACT_TAKESHOT && B.b <= m->host_slots) taken.push_back(B.b);
                    if (B.op != ACT_RESTORE || B.b == 0 || B.b > m->host_slots) continue;
                    if (std::find(taken.begin(), taken.end(), B.b) != taken.end()) continue;
                    const int nb = aj + 1 < acts.size() && acts[aj + 1].op == ACT_YOUTURN ? 1 : 2;
                    bool held = false;
                    for (int q = 0; q < 3; ++q) held |= cx.stage_slot[q] == B.b;
                    for (int q = 0; q < 2; ++q) held |= cx.rest_slot[q] == B.b && cx.rest_fields[q] >= nb;
                    if (held) {
                        if (cx.rest_slot[o] == B.b) break;   // the target pair is needed first
                        continue;
                    }
                    const char* hs = static_cast<const char*>(m->hpool.p) + (size_t)(B.b - 1) * 2 * fb;
                    // after every step issued so far (the pair may still be read by them);
                    // the copy stream has every copy to the host before it
                    CK_TRY(cudaEventRecord(m->ev_fork, cx.st));
                    CK_TRY(cudaStreamWaitEvent(m->side, m->ev_fork, 0));
                    for (int w = 0; w < nb; ++w)
                        CK_TRY(cudaMemcpyAsync(m->hrest[o][w].p, hs + w * fb, fb, cudaMemcpyDefault, m->side));
                    CK_TRY(cudaEventRecord(m->ev_pf[o], m->side));
                    cx.rest_slot[o] = B.b;
                    cx.rest_fields[o] = nb;
                    cx.rest_pf[o] = true;
                    break;
                }
            } else if (rc.mode == CKFWI_STORE_FP32) {
                st = State{slot_r(A.b, 0), slot_r(A.b, 1), U_FP32, U_FP32};   // the slot is the state
            } else if (rc.codec) {
                if (cx.issue) {
                    auto dec = [&](ckfwi_model* m, const long long* from, float* x) -> cudaError_t {
                        if (rc.rate)
                            return codec_rate_decompress_dev(m->pool.as<uint32_t>(), from, m->cap_words,
                                                             field_view(m->fg), rc.rate, x, m->flags.as<int>() + 1,
                                                             cx.st);
                        return codec_decompress_dev(m->pool.as<uint32_t>(), from, m->cap_words, field_view(m->fg), x,
                                                    m->flags.as<int>() + 1, cx.st);
                    };
                    int tok = cx.begin(PC_DECOMP);
                    for (int l = 0; l < NL; ++l) {
                        ckfwi_model* m = cx.lane(l);
                        CK_TRY(dec(m, sbase(m, A.b), cx.fptr(l, work_r(0))));
                        ++cx.launches;
                    }
                    cx.end(tok);
                    if (!next_turn) {   // a reverse step needs u^s only
                        tok = cx.begin(PC_DECOMP);
                        for (int l = 0; l < NL; ++l) {
                            ckfwi_model* m = cx.lane(l);
                            CK_TRY(dec(m, smid(m, A.b), cx.fptr(l, work_r(1))));
                            ++cx.launches;
                        }
                        cx.end(tok);
                    }
                }
                st = State{work_r(0), work_r(1), U_FP32, U_FP32};
            } else if (next_turn) {
                // a reverse step needs u^s only: up-cast that field.  (The
                // reverse kernels can read 16-bit u^s directly, but on this
                // GPU the up-cast plus an FP32 step, whose u^s then comes
                // from L2, is faster: 15 + 80 us against 105 us at 208^3.)
                if (cx.issue) {
                    const int tok = cx.begin(PC_DECOMP);
                    for (int l = 0; l < NL; ++l) {
                        ckfwi_model* m = cx.lane(l);
                        CK_TRY(launch_cast_restore(cx.ptr(l, slot_r(A.b, 0)), ut_slot, m->fg, cx.fptr(l, work_r(0)),
                                                   cx.st));
                        cx.launches += 1;
                    }
                    cx.end(tok);
                }
                st = State{work_r(0), slot_r(A.b, 1), U_FP32, ut_slot};
            } else {
                if (cx.issue) {
                    const int tok = cx.begin(PC_DECOMP);
                    for (int l = 0; l < NL; ++l) {
                        ckfwi_model* m = cx.lane(l);
                        CK_TRY(launch_cast_restore(cx.ptr(l, slot_r(A.b, 0)), ut_slot, m->fg, cx.fptr(l, work_r(0)),
                                                   cx.st));
                        CK_TRY(launch_cast_restore(cx.ptr(l, slot_r(A.b, 1)), ut_slot, m->fg, cx.fptr(l, work_r(1)),
                                                   cx.st));
                        cx.launches += 2;
                    }
                    cx.end(tok);
                }
                st = State{work_r(0), work_r(1), U_FP32, U_FP32};
            }
        } else if (A.op == ACT_YOUTURN) {
            if (first_sweep) {
                // extra step N-1 -> N records d^{N-1}; d^N from u^N
                ST_TRY(fwd_step(cx, st.cur, st.prev, UN_R, N - 1, true, CK_NONE, NONE_R, NONE_R));
                ++fsteps;
                ST_TRY(sample_last(cx, UN_R));
                ST_TRY(field_absmax(cx, UN_R));
                ST_TRY(residual(cx));
                first_sweep = false;
            }
            ST_TRY(reverse(A.a, st.cur, st.tcur));
        }
    }
    // join the copy stream: no checkpoint copy or prefetch outlives the gradient
    if (cx.stage) {
        CK_TRY(cudaEventRecord(cx.m->ev_join, cx.m->side));
        CK_TRY(cudaStreamWaitEvent(cx.st, cx.m->ev_join, 0));
        for (int k = 0; k < 3; ++k) cx.pend[k] = false;
    }
    counters[0] = fsteps;
    counters[1] = ncomp;
    return CKFWI_OK;
}

// Device bytes one lane's checkpoint storage takes for this configuration.
double storage_bytes(const FieldGeom& f, const RunCfg& rc, const ckfwi_grad_opts* o)
{
    if (rc.store_all) return (double)field_bytes(f) * rc.N;
    if (rc.M <= 1) return 0.0;
    const double nslot = (double)(rc.M - 1) * 2;
    if (rc.mode == CKFWI_STORE_FP32) return nslot * field_bytes(f, 4);
    if (!rc.codec) return nslot * field_bytes(f, 2);
    if (rc.rate) return nslot * 4.0 * (double)codec_rate_words(f.dims, f.nz, f.ny, f.nx, rc.rate);
    const double pool = o->pool_bytes ? (double)o->pool_bytes : nslot * f.npts * 4.0;
    return pool + (double)codec_scratch_bytes(f.dims, f.nz, f.ny, f.nx);
}

int prepare_storage(ckfwi_model* m, const RunCfg& rc, const ckfwi_grad_opts* o)
{
    const FieldGeom& f = m->fg;
    const void* before[7] = {m->traj.p, m->pool.p, m->slotbase.p, m->scratch.p, m->statw.p, m->hpool.d,
                             reinterpret_cast<const void*>((intptr_t)m->host_slots)};
    struct Bump {
        ckfwi_model* m;
        const void* const* b;
        ~Bump()
        {
            const void* after[7] = {m->traj.p, m->pool.p, m->slotbase.p, m->scratch.p, m->statw.p, m->hpool.d,
                                    reinterpret_cast<const void*>((intptr_t)m->host_slots)};
            for (int i = 0; i < 7; ++i)
                if (after[i] != b[i]) ++m->gen;
        }
    } bump{m, before};
    m->cap_words = 0;
    m->host_slots = 0;
    if (rc.store_all) {
        CK_TRY(m->traj.alloc(field_bytes(f) * (size_t)rc.N));
        return CKFWI_OK;
    }
    if (rc.M <= 1) return CKFWI_OK;
    // Uncompressed slots are read with their halo cells, which must hold 0;
    // a pool last used with another layout is cleared before reuse.
    const int tag = rc.mode == CKFWI_STORE_FP32 ? 4 : (rc.codec ? 0 : 2);
    if (!rc.codec) {
        // the first host_slots slots in pinned host memory, the others on the device
        const int hs = std::max(0, std::min(o->host_slots, rc.M - 1));
        const size_t dslot = (size_t)(rc.M - 1 - hs) * 2, hslot = (size_t)hs * 2;
        const size_t need = dslot * field_bytes(f, (size_t)tag);
        const void* before_p = m->pool.p;
        const int old_tag = m->pool_tag;
        CK_TRY(m->pool.alloc(need));
        if (m->pool.p == before_p && old_tag != tag && m->pool.p) {
            CK_TRY(cudaMemset(m->pool.p, 0, m->pool.bytes));
            CK_TRY(cudaDeviceSynchronize());
        }
        if (hs > 0) {
            const void* before_h = m->hpool.p;
            CK_TRY(m->hpool.alloc(hslot * field_bytes(f, (size_t)tag)));
            if (m->hpool.p == before_h && old_tag != tag) std::memset(m->hpool.p, 0, m->hpool.bytes);
        } else if (m->hpool.p && old_tag != tag) {
            std::memset(m->hpool.p, 0, m->hpool.bytes);
        }
        m->host_slots = hs;
        m->pool_tag = tag;
        if (hs > 0 && tag == 4) {
            // the staging pairs and the copy stream of FP32 host slots
            for (int k = 0; k < 3; ++k)
                for (int w = 0; w < 2; ++w) CK_TRY(m->hstage[k][w].alloc(field_bytes(f)));
            for (int r = 0; r < 2; ++r)
                for (int w = 0; w < 2; ++w) CK_TRY(m->hrest[r][w].alloc(field_bytes(f)));
            if (!m->side) CK_TRY(cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking));
            if (!m->ev_fork) CK_TRY(cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming));
            for (int k = 0; k < 3; ++k)
                if (!m->ev_done[k]) CK_TRY(cudaEventCreateWithFlags(&m->ev_done[k], cudaEventDisableTiming));
            for (int r = 0; r < 2; ++r)
                if (!m->ev_pf[r]) CK_TRY(cudaEventCreateWithFlags(&m->ev_pf[r], cudaEventDisableTiming));
            if (!m->ev_join) CK_TRY(cudaEventCreateWithFlags(&m->ev_join, cudaEventDisableTiming));
        }
    } else {
        m->pool_tag = 0;
        size_t bytes = o->pool_bytes ? o->pool_bytes : (size_t)(rc.M - 1) * 2 * f.npts * 4;
        if (rc.rate) {
            // fixed-rate streams: the exact size is known, a smaller budget is refused up front
            const size_t need = (size_t)(rc.M - 1) * 2 * 4 * (size_t)codec_rate_words(f.dims, f.nz, f.ny, f.nx, rc.rate);
            if (o->pool_bytes && o->pool_bytes < need) return CKFWI_EINVAL;
            bytes = need;
        }
        bytes = (bytes + 3) / 4 * 4;
        CK_TRY(m->pool.alloc(bytes, false));
        m->cap_words = (long long)(bytes / 4);
        CK_TRY(m->slotbase.alloc(sizeof(long long) * (2 * (size_t)rc.M + 4)));
        // a fresh scratch is zeroed (its counter and group sums start at zero;
        // every compression of this model's fields leaves them zero)
        if (!rc.rate) CK_TRY(m->scratch.alloc((size_t)codec_scratch_bytes(f.dims, f.nz, f.ny, f.nx), true));
        CK_TRY(m->statw.alloc(sizeof(unsigned long long) * (size_t)(4 * rc.N + 8)));
    }
    return CKFWI_OK;
}

float tol_float(double tol)
{
    float t = (float)tol;
    if ((double)t > tol) t = std::nextafter(t, 0.0f);
    return t;
}

int check_opts(const ckfwi_grad_opts* o)
{
    if (!o) return CKFWI_EINVAL;
    if (o->ckpt_slots < 1) return CKFWI_EINVAL;
    if (o->store_mode < 0 || o->store_mode > 4) return CKFWI_EINVAL;
    if (o->store_mode == CKFWI_STORE_CODEC_RATE && (o->rate < 1 || o->rate > 32)) return CKFWI_EINVAL;
    if (o->grad_kind != CKFWI_VELOCITY && o->grad_kind != CKFWI_SLOWNESS2) return CKFWI_EINVAL;
    if (o->store_mode == CKFWI_STORE_CODEC && (!(o->tol >= std::ldexp(1.0, -90)) || !std::isfinite(o->tol)))
        return CKFWI_EINVAL;
    return CKFWI_OK;
}

RunCfg run_cfg(int nt, const ckfwi_grad_opts* o)
{
    RunCfg rc{};
    rc.N = nt;
    rc.M = o->ckpt_slots;
    rc.mode = o->store_mode;
    rc.codec = rc.mode == CKFWI_STORE_CODEC || rc.mode == CKFWI_STORE_CODEC_RATE;
    rc.rate = rc.mode == CKFWI_STORE_CODEC_RATE ? o->rate : 0;
    rc.tol_f = rc.mode == CKFWI_STORE_CODEC ? tol_float(o->tol) : (float)rc.rate;
    rc.store_all = rc.M >= rc.N && rc.mode == CKFWI_STORE_FP32;
    if (rc.M > rc.N) rc.M = rc.N;
    return rc;
}

// Keep at most `cap` recorded graphs per model (oldest recorded first out).
template <class Map>
void trim_graphs(Map& g, std::vector<typename Map::key_type>& order, size_t cap)
{
    while (order.size() > cap) {
        auto it = g.find(order.front());
        if (it != g.end()) {
            it->second.release();
            g.erase(it);
        }
        order.erase(order.begin());
    }
}

// Fill stats from the per-class timings and the schedule counts.
// the float max |u| that field_absmax left in the low word of a double slot
double absmax_of(double slot)
{
    uint32_t b = 0;
    std::memcpy(&b, &slot, sizeof(b));
    float f = 0.0f;
    std::memcpy(&f, &b, sizeof(f));
    return (double)f;
}

void fill_stats(ckfwi_stats* stats, Ctx& cx, const RunCfg& rc, const long long* cnt, const long long* counters,
                const FieldGeom& f)
{
    std::memset(stats, 0, sizeof(*stats));
    const Tile tf = cx.batch ? cx.bf : cx.m->tf, ta = cx.batch ? cx.ba : cx.m->ta;
    stats->fwd_ver = tf.ver;
    stats->fwd_bx = tf.bx;
    stats->fwd_by = tf.by;
    stats->fwd_vec = tf.vec;
    stats->fwd_zlen = cx.batch ? cx.zf[0] : tf.zlen;
    stats->adj_ver = ta.ver;
    stats->adj_bx = ta.bx;
    stats->adj_by = ta.by;
    stats->adj_vec = ta.vec;
    stats->adj_zlen = cx.batch ? cx.za[0] : ta.zlen;
    stats->fwd_pf = tf.pf;
    stats->adj_pf = ta.pf;
    stats->fwd_steps = counters[0];
    stats->adj_steps = rc.N;
    stats->p = rc.store_all ? rc.N - 1 : cnt[0];
    stats->takeshots = rc.store_all ? rc.N - 1 : cnt[1];
    stats->restores = rc.store_all ? rc.N - 1 : cnt[2];
    stats->kernel_launches = cx.launches;
    stats->fwd_launches = cx.count[PC_FWD];
    stats->adj_launches = cx.count[PC_ADJ];
    stats->comp_calls = cx.count[PC_COMP];
    stats->decomp_calls = cx.count[PC_DECOMP];
    if (cx.prof.on) {
        double ms[PC_N] = {0, 0, 0, 0, 0};
        for (auto& mk : cx.prof.marks) {
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, (*cx.prof.pool)[mk.second], (*cx.prof.pool)[mk.second + 1]) == cudaSuccess)
                ms[mk.first] += t;
        }
        stats->fwd_ms = ms[PC_FWD];
        stats->adj_ms = ms[PC_ADJ];
        stats->comp_ms = ms[PC_COMP];
        stats->decomp_ms = ms[PC_DECOMP];
        stats->other_ms = ms[PC_OTHER];
    }
    if (rc.store_all) stats->pool_bytes_peak = (double)field_bytes(f) * rc.N;
    else if (rc.mode == CKFWI_STORE_FP32) stats->pool_bytes_peak = (double)(rc.M - 1) * 2 * field_bytes(f, 4);
    else if (!rc.codec) stats->pool_bytes_peak = (double)(rc.M - 1) * 2 * field_bytes(f, 2);
}

// Compression ratios and the peak pool height of one lane's codec run
// (replaying the slot stack with the measured stream sizes).
void codec_stats(const std::vector<long long>& words, const std::vector<Action>& acts, int M, const FieldGeom& f,
                 double* rmin, double* rsum, double* peak_bytes)
{
    const long long ncomp = (long long)words.size();
    double mn = 1e300, sum = 0;
    for (long long wds : words) {
        const double r = (double)f.npts / (double)std::max<long long>(1, wds);
        mn = std::min(mn, r);
        sum += r;
    }
    std::vector<long long> height((size_t)M + 2, 0);
    long long k = 0, peak = 0;
    for (const Action& A : acts) {
        if (A.op != ACT_TAKESHOT || k + 1 >= ncomp) continue;
        height[A.b] = height[A.b - 1] + words[k] + words[k + 1];
        peak = std::max(peak, height[A.b]);
        k += 2;
    }
    *rmin = mn;
    *rsum = sum;
    *peak_bytes = (double)peak * 4;
}

// The action list: Revolve, or with FP32 slots in host memory the two-level
// (multistage) schedule, which writes each host slot once
void make_schedule(const ckfwi_model* m, const RunCfg& rc, std::vector<Action>& acts, long long cnt[3])
{
    if (rc.store_all) return;
    if (rc.mode == CKFWI_STORE_FP32 && !rc.codec && m->host_slots > 0)
        multistage_schedule(rc.N, rc.M, m->host_slots, acts, cnt);
    else
        revolve_schedule(rc.N, rc.M, acts, cnt);
}

int gradient_one(ckfwi_model* m, const ckfwi_shot* s, const float* d_obs, int mem,
                 const ckfwi_grad_opts* o, double* misfit, ckfwi_stats* stats, cudaStream_t st)
{
    if (!m->have_model) return CKFWI_EINVAL;
    if (!d_obs) return CKFWI_EINVAL;
    ST_TRY(check_opts(o));
    ST_TRY(set_shot(m, s));
    ST_TRY(autotune(m, st));
    const FieldGeom& f = m->fg;
    const RunCfg rc = run_cfg(m->g.nt, o);
    ST_TRY(prepare_storage(m, rc, o));
    const size_t nd = (size_t)(rc.N + 1) * m->shot.nrec;
    CK_TRY(cudaMemcpyAsync(m->shot.dobs.p, d_obs, nd * sizeof(float),
                           mem == CKFWI_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    ST_TRY(reset_flags(m, st));
    std::vector<Action> acts;
    long long cnt[3] = {rc.N - 1, 0, 0};
    make_schedule(m, rc, acts, cnt);
    Ctx cx{m, st, 0};
    cx.mode = rc.mode;
    cx.stage = rc.mode == CKFWI_STORE_FP32 && !rc.codec && !rc.store_all && m->host_slots > 0 && m->side;
    long long counters[2] = {0, 0};
    const bool graph = o->use_graph != 0 && !o->profile;
    if (o->profile) {
        cx.prof.on = true;
        cx.prof.pool = &m->evpool;
    }
    GraphKey key{rc.N, rc.M, rc.mode, o->grad_kind, rc.tol_f, (size_t)m->cap_words, m->gen};
    if (graph) {
        auto it = m->graphs.find(key);
        if (it == m->graphs.end()) {
            // record on a private non-blocking stream (the caller's may be the
            // legacy stream, which cannot be captured); replay on the caller's
            if (!m->cap) CK_TRY(cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking));
            CK_TRY(cudaStreamSynchronize(st));
            cudaGraph_t gr;
            cx.st = m->cap;
            CK_TRY(cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeRelaxed));
            const int rs = run_body(cx, rc, acts, counters);
            cudaError_t ee = cudaStreamEndCapture(m->cap, &gr);
            cx.st = st;
            if (rs != CKFWI_OK) {
                if (ee == cudaSuccess) cudaGraphDestroy(gr);
                return rs;
            }
            CK_TRY(ee);
            GraphExec& ge = m->graphs[key];
            cudaError_t ei = cudaGraphInstantiate(&ge.ex, gr, 0);
            cudaGraphDestroy(gr);
            if (ei != cudaSuccess) {
                m->graphs.erase(key);
                return cuda_status(ei);
            }
            ge.launches = cx.launches;
            std::memcpy(ge.count, cx.count, sizeof(cx.count));
            m->graph_order.push_back(key);
            trim_graphs(m->graphs, m->graph_order, MAX_GRAPHS);
            it = m->graphs.find(key);
        } else {
            // the same schedule: counters from a dry count
            counters[0] = rc.store_all ? rc.N : cnt[0] + 1;
            counters[1] = rc.codec ? 2 * cnt[1] : 0;
            cx.launches = it->second.launches;
            std::memcpy(cx.count, it->second.count, sizeof(cx.count));
        }
        CK_TRY(cudaGraphLaunch(it->second.ex, st));
    } else {
        ST_TRY(run_body(cx, rc, acts, counters));
    }
    double phi2[2] = {0.0, 0.0};
    CK_TRY(cudaMemcpyAsync(phi2, m->phi.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    int fl = 0;
    ST_TRY(read_flags(m, st, &fl));
    const double phi = phi2[0];
    if (misfit) *misfit = phi;
    m->last_words.clear();
    if (counters[1] > 0) {
        m->last_words.resize((size_t)counters[1]);
        CK_TRY(cudaMemcpy(m->last_words.data(), m->statw.p, sizeof(long long) * counters[1], cudaMemcpyDeviceToHost));
    }
    if (stats) {
        fill_stats(stats, cx, rc, cnt, counters, f);
        stats->u_absmax = absmax_of(phi2[1]);
        const long long ncomp = counters[1];
        if (ncomp > 0) {
            double mn, sum, peak;
            codec_stats(m->last_words, acts, rc.M, f, &mn, &sum, &peak);
            stats->ratio_min = mn;
            stats->ratio_mean = sum / (double)ncomp;
            stats->pool_bytes_peak = peak;
        }
    }
    return fl;
}

// ------------------------------------------------------------ batched shots
long long lane_blocks(const FieldGeom& f, const Tile& t, int zlen)
{
    const long long gx = (f.nx + t.bx - 1) / t.bx;
    const long long gy = f.dims == 3 ? (f.ny + t.by - 1) / t.by : 1;
    return gx * gy * ((f.nz + zlen - 1) / zlen);
}

// CTA offsets of the lanes in a batched launch (lanes + 1 entries)
std::vector<int> lane_starts(const std::vector<ckfwi_model*>& lanes, const Tile& t, const std::vector<int>& z,
                             long long* total)
{
    std::vector<int> s(lanes.size() + 1, 0);
    long long acc = 0;
    for (size_t l = 0; l < lanes.size(); ++l) {
        s[l] = (int)std::min<long long>(acc, 0x7fffffffLL);
        acc += lane_blocks(lanes[l]->fg, t, z[l]);
    }
    s[lanes.size()] = (int)std::min<long long>(acc, 0x7fffffffLL);
    *total = acc;
    return s;
}

std::vector<long long> lane_ids(const std::vector<ckfwi_model*>& lanes, bool with_gen)
{
    std::vector<long long> v;
    for (ckfwi_model* L : lanes) {
        v.push_back(L->uid);
        if (with_gen) v.push_back(L->gen);
    }
    return v;
}

// Batch autotuner: a common tile shape and a z-run length per lane, picked
// by timing batched forward and reverse launches over all lanes.  The
// candidates split every column into nzc runs, nzc chosen so that the
// whole batch has 1 to 16 CTAs per SM.
int batch_tune(const std::vector<ckfwi_model*>& lanes, cudaStream_t st, const BatchTiles** out)
{
    ckfwi_model* m0 = lanes[0];
    const std::vector<long long> key = lane_ids(lanes, false);
    auto it = m0->btiles.find(key);
    if (it != m0->btiles.end()) {
        *out = &it->second;
        return CKFWI_OK;
    }
    const int dims = m0->fg.dims, K = m0->K, NL = (int)lanes.size();
    int dev = 0, nsm = 0;
    CK_TRY(cudaGetDevice(&dev));
    CK_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    struct Cand {
        Tile t;
        std::vector<int> z;
    };
    std::vector<Cand> cands;
    std::vector<Tile> shapes;
    for (int i = 0; i < tile_count(dims); ++i) {
        const Tile t = tile_at(dims, i, 1);
        if (tile_supported(dims, K, t)) shapes.push_back(t);
    }
    bool fits3 = dims == 3;
    for (ckfwi_model* L : lanes) fits3 = fits3 && v3_fits(L->fg, K);
    for (int i = 0; fits3 && i < v3_shape_count(); ++i) {
        const Tile t = v3_tile_at(i, 1);
        if (v3_supported(dims, K, t)) shapes.push_back(t);
        if (t.vec != 4) continue;
        Tile t4 = t;                     // fed by asynchronous copies (forward step only)
        t4.ver = 4;
        t4.pf = K <= 4 ? 1 : 2;
        if (v4_supported(dims, K, t4)) shapes.push_back(t4);
        Tile t7 = t;                     // the lean generation, one or two planes per step
        t7.ver = 7;
        for (int np : {1, 2}) {
            t7.pf = np;
            if (v5_supported(dims, K, t7)) shapes.push_back(t7);
        }
    }
    // CKFWI_BATCH_VER restricts the timed candidates to one generation
    // (tests); generation 4 has no batched reverse step, which then takes
    // the vector-blocked kernels
    const char* bv = std::getenv("CKFWI_BATCH_VER");
    const int want = bv ? std::atoi(bv) : 0;
    for (const Tile& t : shapes) {
        long long cols = 0;
        int nzmax = 1;
        for (ckfwi_model* L : lanes) {
            cols += (long long)((L->fg.nx + t.bx - 1) / t.bx) * (dims == 3 ? (L->fg.ny + t.by - 1) / t.by : 1);
            nzmax = std::max(nzmax, L->fg.nz);
        }
        std::vector<std::vector<int>> seen;
        for (int target : {1, 2, 4, 8, 16}) {
            long long nzc = (target * (long long)nsm + cols - 1) / cols;
            nzc = std::max<long long>(1, std::min<long long>(nzc, nzmax));
            std::vector<int> z(NL);
            for (int l = 0; l < NL; ++l) z[l] = std::max(4, (int)((lanes[l]->fg.nz + nzc - 1) / nzc));
            if (std::find(seen.begin(), seen.end(), z) != seen.end()) continue;
            seen.push_back(z);
            cands.push_back(Cand{t, z});
        }
    }
    if (cands.empty()) return CKFWI_EINVAL;
    // argument tables of a probe step on the lanes' own working buffers
    std::vector<FwdArgs> fa(NL);
    std::vector<AdjArgs> aa(NL);
    for (int l = 0; l < NL; ++l) {
        ckfwi_model* L = lanes[l];
        const FieldGeom& f = L->fg;
        fa[l] = fwd_args(L);
        fa[l].u = org(L->work[0], f);
        fa[l].up = org(L->work[1], f);
        fa[l].out = org(L->work[2], f);
        fa[l].src = L->shot.src.view;
        fa[l].src.series = L->shot.wavelet.as<float>();
        aa[l] = adj_args(L);
        aa[l].l1 = org(L->lam[0], f);
        aa[l].l2 = org(L->lam[1], f);
        aa[l].l0 = org(L->lam[2], f);
        aa[l].u = org(L->work[0], f);
        aa[l].adj = L->shot.adj.view;
        aa[l].adj.series = L->shot.resid.as<float>();
        aa[l].src = L->shot.src.view;
        aa[l].src.series = L->shot.wavelet.as<float>();
    }
    DevMem dtab, dst;
    CK_TRY(dtab.alloc(sizeof(FwdArgs) * NL + sizeof(AdjArgs) * NL + 256, false));
    CK_TRY(dst.alloc(sizeof(int) * (NL + 1), false));
    FwdArgs* ftab = dtab.as<FwdArgs>();
    AdjArgs* atab = reinterpret_cast<AdjArgs*>(dtab.as<char>() + ((sizeof(FwdArgs) * NL + 255) / 256) * 256);
    cudaEvent_t e0, e1;
    CK_TRY(cudaEventCreate(&e0));
    CK_TRY(cudaEventCreate(&e1));
    const bool verbose = std::getenv("CKFWI_VERBOSE") != nullptr;
    float best[2] = {1e30f, 1e30f};
    bool warmed = false;
    BatchTiles bt;
    int rs = CKFWI_OK;
    for (const Cand& c : cands) {
        long long total = 0;
        const std::vector<int> s = lane_starts(lanes, c.t, c.z, &total);
        if (total > 0x7fffffffLL) continue;
        for (int l = 0; l < NL; ++l) {
            fa[l].zlen = c.z[l];
            aa[l].zlen = c.z[l];
        }
        if (cudaMemcpy(ftab, fa.data(), sizeof(FwdArgs) * NL, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(atab, aa.data(), sizeof(AdjArgs) * NL, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(dst.p, s.data(), sizeof(int) * (NL + 1), cudaMemcpyHostToDevice) != cudaSuccess) {
            rs = CKFWI_ECUDA;
            break;
        }
        for (int pass = 0; pass < 2 && rs == CKFWI_OK; ++pass) {
            if (pass == 1 && c.t.ver == 4) continue;    // generation 4 has no batched reverse step
            if (want && c.t.ver != want && !(want == 4 && pass == 1 && c.t.ver == 3)) continue;
            auto go = [&]() {
                const BatchLaunch<FwdArgs> bf{ftab, dst.as<int>(), NL, dims, total};
                const BatchLaunch<AdjArgs> ba{atab, dst.as<int>(), NL, dims, total};
                if (c.t.ver == 7)
                    return pass == 0 ? launch_fwd5_batch(bf, c.t, K, CK_NONE, st)
                                     : launch_adj5_batch(ba, c.t, K, U_FP32, st);
                if (c.t.ver == 4) return launch_fwd4_batch(bf, c.t, K, CK_NONE, st);
                if (c.t.ver == 3)
                    return pass == 0 ? launch_fwd3_batch(bf, c.t, K, CK_NONE, st)
                                     : launch_adj3_batch(ba, c.t, K, U_FP32, st);
                return pass == 0 ? launch_fwd_batch(bf, c.t, K, CK_NONE, st)
                                 : launch_adj_batch(ba, c.t, K, U_FP32, st);
            };
            const int reps = 3;
            // the first candidate also brings the clocks up; then the median of three timings
            cudaError_t e = cudaSuccess;
            for (int r = 0; r < (warmed ? 1 : 20) && e == cudaSuccess; ++r) e = go();
            std::vector<float> v;
            for (int round = 0; round < 3 && e == cudaSuccess; ++round) {
                e = cudaEventRecord(e0, st);
                for (int r = 0; r < reps && e == cudaSuccess; ++r) e = go();
                if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float t = 0;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
                v.push_back(t);
            }
            if (e != cudaSuccess) {
                rs = cuda_status(e);
                break;
            }
            warmed = true;
            std::sort(v.begin(), v.end());
            const float ms = v[1];
            if (verbose)
                std::fprintf(stderr, "ckfwi batch autotune %s lanes %d ver %d tile %dx%d vec %d z[0] %d: %.1f us\n",
                             pass ? "adj" : "fwd", NL, c.t.ver, c.t.bx, c.t.by, c.t.vec, c.z[0],
                             1000.0f * ms / reps);
            if (ms < best[pass]) {
                best[pass] = ms;
                if (pass == 0) {
                    bt.tf = c.t;
                    bt.zf = c.z;
                } else {
                    bt.ta = c.t;
                    bt.za = c.z;
                }
            }
        }
        if (rs != CKFWI_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ST_TRY(rs);
    if (bt.zf.empty() || bt.za.empty()) return CKFWI_EINVAL;
    // the probes wrote into working buffers; clear them
    for (ckfwi_model* L : lanes) {
        for (int i = 0; i < 3; ++i) {
            CK_TRY(cudaMemsetAsync(L->work[i].p, 0, L->work[i].bytes, st));
            CK_TRY(cudaMemsetAsync(L->lam[i].p, 0, L->lam[i].bytes, st));
        }
        CK_TRY(cudaMemsetAsync(L->gacc.p, 0, L->gacc.bytes, st));
    }
    CK_TRY(cudaStreamSynchronize(st));
    auto ins = m0->btiles.emplace(key, std::move(bt)).first;
    *out = &ins->second;
    return CKFWI_OK;
}

// Misfits (phis[l]) and gradients (left in each lane's gacc) of one batch:
// lane l runs shots[l] on model lanes[l], all lanes through one Revolve
// schedule, every stencil step one launch over all lanes.  Lanes may have
// different grids (apertures); they share dims, space order and nt.
int gradient_batch(const std::vector<ckfwi_model*>& lanes, const ckfwi_shot* shots, const float* const* d_obs,
                   int mem, const ckfwi_grad_opts* o, double* phis, ckfwi_stats* stats, cudaStream_t st)
{
    ST_TRY(check_opts(o));
    const int NL = (int)lanes.size();
    ckfwi_model* m0 = lanes[0];
    for (int l = 0; l < NL; ++l) {
        ckfwi_model* L = lanes[l];
        if (!L->have_model || !d_obs[l]) return CKFWI_EINVAL;
        if (L->fg.dims != m0->fg.dims || L->K != m0->K || L->g.nt != m0->g.nt) return CKFWI_EINVAL;
    }
    for (int l = 0; l < NL; ++l) ST_TRY(set_shot(lanes[l], shots + l));
    const RunCfg rc = run_cfg(m0->g.nt, o);
    for (int l = 0; l < NL; ++l) ST_TRY(prepare_storage(lanes[l], rc, o));
    const BatchTiles* bt = nullptr;
    ST_TRY(batch_tune(lanes, st, &bt));
    for (int l = 0; l < NL; ++l) {
        ckfwi_model* L = lanes[l];
        const size_t nd = (size_t)(rc.N + 1) * L->shot.nrec;
        CK_TRY(cudaMemcpyAsync(L->shot.dobs.p, d_obs[l], nd * sizeof(float),
                               mem == CKFWI_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
        ST_TRY(reset_flags(L, st));
    }
    std::vector<Action> acts;
    long long cnt[3] = {rc.N - 1, 0, 0};
    make_schedule(m0, rc, acts, cnt);
    Ctx cx{m0, st, 0};
    cx.mode = rc.mode;
    cx.lanes = lanes;
    cx.batch = true;
    cx.bf = bt->tf;
    cx.ba = bt->ta;
    cx.zf = bt->zf;
    cx.za = bt->za;
    const std::vector<int> fs = lane_starts(lanes, cx.bf, cx.zf, &cx.fblocks);
    const std::vector<int> as = lane_starts(lanes, cx.ba, cx.za, &cx.ablocks);
    if (cx.fblocks > 0x7fffffffLL || cx.ablocks > 0x7fffffffLL) return CKFWI_EINVAL;
    long long counters[2] = {0, 0};
    const bool graph = o->use_graph != 0 && !o->profile;
    if (o->profile) {
        cx.prof.on = true;
        cx.prof.pool = &m0->evpool;
    }
    BatchKey key{lane_ids(lanes, true), rc.N, rc.M, rc.mode, o->grad_kind, rc.tol_f};
    auto it = graph ? m0->bgraphs.find(key) : m0->bgraphs.end();
    if (it != m0->bgraphs.end()) {
        counters[0] = rc.store_all ? rc.N : cnt[0] + 1;
        counters[1] = rc.codec ? 2 * cnt[1] : 0;
        cx.launches = it->second.ex.launches;
        std::memcpy(cx.count, it->second.ex.count, sizeof(cx.count));
        CK_TRY(cudaGraphLaunch(it->second.ex.ex, st));
    } else {
        // pass 1: collect every step's per-lane arguments
        cx.issue = false;
        ST_TRY(run_body(cx, rc, acts, counters));
        // the tables live with the graph that reads them, or in scratch
        BatchGraph tmp;
        BatchGraph& bg = graph ? m0->bgraphs[key] : tmp;
        DevMem& tabs = graph ? bg.tabs : m0->btabs;
        const size_t fb = ((sizeof(FwdArgs) * cx.ftab.size() + 255) / 256) * 256;
        const size_t ab = ((sizeof(AdjArgs) * cx.atab.size() + 255) / 256) * 256;
        const size_t sb = sizeof(int) * 2 * (NL + 1);
        int rs = cuda_status_or_ok(tabs.alloc(fb + ab + sb, false));
        if (rs == CKFWI_OK && !cx.ftab.empty())
            rs = cuda_status_or_ok(cudaMemcpy(tabs.p, cx.ftab.data(), sizeof(FwdArgs) * cx.ftab.size(),
                                              cudaMemcpyHostToDevice));
        if (rs == CKFWI_OK && !cx.atab.empty())
            rs = cuda_status_or_ok(cudaMemcpy(tabs.as<char>() + fb, cx.atab.data(),
                                              sizeof(AdjArgs) * cx.atab.size(), cudaMemcpyHostToDevice));
        std::vector<int> starts(fs);
        starts.insert(starts.end(), as.begin(), as.end());
        if (rs == CKFWI_OK)
            rs = cuda_status_or_ok(
                cudaMemcpy(tabs.as<char>() + fb + ab, starts.data(), sb, cudaMemcpyHostToDevice));
        if (rs != CKFWI_OK) {
            if (graph) m0->bgraphs.erase(key);
            return rs;
        }
        cx.ftab_d = tabs.as<FwdArgs>();
        cx.atab_d = reinterpret_cast<const AdjArgs*>(tabs.as<char>() + fb);
        cx.fstart_d = reinterpret_cast<const int*>(tabs.as<char>() + fb + ab);
        cx.astart_d = cx.fstart_d + (NL + 1);
        cx.fi = cx.ai = 0;
        cx.issue = true;
        // pass 2: issue (recorded into a graph when asked)
        if (graph) {
            if (!m0->cap) rs = cuda_status_or_ok(cudaStreamCreateWithFlags(&m0->cap, cudaStreamNonBlocking));
            if (rs == CKFWI_OK) rs = cuda_status_or_ok(cudaStreamSynchronize(st));
            cudaGraph_t gr = nullptr;
            if (rs == CKFWI_OK) {
                Ctx& cc = cx;
                cc.st = m0->cap;
                rs = cuda_status_or_ok(cudaStreamBeginCapture(m0->cap, cudaStreamCaptureModeRelaxed));
                if (rs == CKFWI_OK) {
                    const int rb = run_body(cc, rc, acts, counters);
                    const cudaError_t ee = cudaStreamEndCapture(m0->cap, &gr);
                    rs = rb != CKFWI_OK ? rb : cuda_status_or_ok(ee);
                    if (rb != CKFWI_OK && ee == cudaSuccess) cudaGraphDestroy(gr);
                }
                cc.st = st;
            }
            if (rs == CKFWI_OK) {
                rs = cuda_status_or_ok(cudaGraphInstantiate(&bg.ex.ex, gr, 0));
                cudaGraphDestroy(gr);
            }
            if (rs != CKFWI_OK) {
                m0->bgraphs.erase(key);
                return rs;
            }
            bg.ex.launches = cx.launches;
            std::memcpy(bg.ex.count, cx.count, sizeof(cx.count));
            m0->bgraph_order.push_back(key);
            trim_graphs(m0->bgraphs, m0->bgraph_order, MAX_GRAPHS);
            CK_TRY(cudaGraphLaunch(m0->bgraphs[key].ex.ex, st));
        } else {
            ST_TRY(run_body(cx, rc, acts, counters));
        }
    }
    int fl = 0;
    double umax = 0.0;
    for (int l = 0; l < NL; ++l) {
        double p2[2] = {0.0, 0.0};
        CK_TRY(cudaMemcpyAsync(p2, lanes[l]->phi.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        int f1 = 0;
        ST_TRY(read_flags(lanes[l], st, &f1));
        phis[l] = p2[0];
        umax = std::max(umax, absmax_of(p2[1]));
        if (fl == CKFWI_OK) fl = f1;
    }
    if (stats) {
        fill_stats(stats, cx, rc, cnt, counters, m0->fg);
        stats->u_absmax = umax;
        const long long ncomp = counters[1];
        if (ncomp > 0) {
            double mn = 1e300, sum = 0, peak = 0;
            for (int l = 0; l < NL; ++l) {
                std::vector<long long> words(ncomp);
                CK_TRY(cudaMemcpy(words.data(), lanes[l]->statw.p, sizeof(long long) * ncomp,
                                  cudaMemcpyDeviceToHost));
                double a, b, c;
                codec_stats(words, acts, rc.M, lanes[l]->fg, &a, &b, &c);
                mn = std::min(mn, a);
                sum += b;
                peak = std::max(peak, c);
            }
            stats->ratio_min = mn;
            stats->ratio_mean = sum / (double)(ncomp * NL);
            stats->pool_bytes_peak = peak;
        } else {
            double peak = 0;
            for (ckfwi_model* L : lanes) peak = std::max(peak, storage_bytes(L->fg, rc, o));
            stats->pool_bytes_peak = peak;
        }
    }
    return fl;
}

// Clones of a model: extra lanes with the same grid and medium, so that
// several shots on one model can run as one batch.
int ensure_clones(ckfwi_model* m, int k, cudaStream_t st)
{
    while ((int)m->clones.size() < k) {
        ckfwi_model* c = nullptr;
        ST_TRY(ckfwi_create_model(&m->g, &c));
        m->clones.emplace_back(c);
    }
    for (int i = 0; i < k; ++i) {
        ckfwi_model* c = m->clones[i].get();
        if (c->src_ver == m->model_ver && c->have_model) continue;
        CK_TRY(cudaMemcpyAsync(c->w.p, m->w.p, m->w.bytes, cudaMemcpyDeviceToDevice, st));
        CK_TRY(cudaMemcpyAsync(c->cvel.p, m->cvel.p, m->cvel.bytes, cudaMemcpyDeviceToDevice, st));
        c->have_model = true;
        c->src_ver = m->model_ver;
    }
    CK_TRY(cudaStreamSynchronize(st));
    return CKFWI_OK;
}

// How many shots of one model run side by side: bounded by free device
// memory (a lane holds ten fields and its checkpoint storage), by
// CKFWI_MAX_LANES (default 64) and by the shot count.
int batch_width(ckfwi_model* m, int nshots, const ckfwi_grad_opts* o)
{
    if (m->ot == 4) return 1;     // the OT4 kernels have no batched form: one shot at a time
    int cap = 64;
    if (const char* v = std::getenv("CKFWI_MAX_LANES")) cap = std::max(1, std::atoi(v));
    const RunCfg rc = run_cfg(m->g.nt, o);
    const double lane = 10.0 * field_bytes(m->fg) + 8.0 * m->fg.npts + storage_bytes(m->fg, rc, o);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return 1;
    const double extra = 0.8 * (double)fr / lane;
    const long long w = 1 + (long long)m->clones.size() + (long long)extra;
    return (int)std::max<long long>(1, std::min<long long>({(long long)nshots, (long long)cap, w}));
}

}  // namespace

extern "C" {

int ckfwi_create_model(const ckfwi_grid* g, ckfwi_model** out)
{
    if (!out) return CKFWI_EINVAL;
    *out = nullptr;
    ST_TRY(check_grid(g));
    ckfwi_model* m = new (std::nothrow) ckfwi_model();
    if (!m) return CKFWI_ENOMEM;
    std::unique_ptr<ckfwi_model> guard(m);
    static std::atomic<long long> next_uid{1};
    m->uid = next_uid++;
    m->g = *g;
    if (g->dims == 2) m->g.n[1] = 1;
    m->K = g->space_order / 2;
    m->fg = make_geom(g->dims, g->n[0], m->g.n[1], g->n[2], m->K);
    // CKFWI_TMA_WAIT_LIMIT < 0 makes the TMA kernels' waits run out at once
    // (the test of the CKFWI_TIMEOUT path; the copies in flight are still
    // waited for before a CTA leaves)
    if (const char* wl = std::getenv("CKFWI_TMA_WAIT_LIMIT")) m->wait_limit = std::atoll(wl);
    double c[MAXK + 1];
    fd_weights(m->K, c);
    const double ih2 = 1.0 / (g->h * g->h);
    m->c[0] = 0.0f;   // the difference-form Laplacian needs c_j, j >= 1, only
    for (int j = 1; j <= m->K; ++j) m->c[j] = (float)(c[j] * ih2);
    m->ot = g->time_order == 4 ? 4 : 2;
    for (int j = 1; j <= m->K; ++j) m->c12[j] = (float)(c[j] * ih2 / 12.0);
    m->hdt = (float)(g->dt / 2.0);
    const FieldGeom& f = m->fg;
    std::vector<float> eta((size_t)f.nz + f.ny + f.nx);
    for (int i = 0; i < f.nz; ++i) eta[i] = (float)eta_axis(m->g, i, f.nz);
    for (int i = 0; i < f.ny; ++i) eta[f.nz + i] = g->dims == 3 ? (float)eta_axis(m->g, i, f.ny) : 0.0f;
    for (int i = 0; i < f.nx; ++i) eta[f.nz + f.ny + i] = (float)eta_axis(m->g, i, f.nx);
    CK_TRY(m->eta.alloc(eta.size() * sizeof(float), false));
    CK_TRY(cudaMemcpy(m->eta.p, eta.data(), eta.size() * sizeof(float), cudaMemcpyHostToDevice));
    CK_TRY(m->w.alloc(field_bytes(f)));
    CK_TRY(m->cvel.alloc((size_t)f.npts * sizeof(float)));
    CK_TRY(m->zero.alloc(field_bytes(f)));
    CK_TRY(m->uN.alloc(field_bytes(f)));
    for (int i = 0; i < 3; ++i) {
        CK_TRY(m->work[i].alloc(field_bytes(f)));
        CK_TRY(m->lam[i].alloc(field_bytes(f)));
    }
    CK_TRY(m->gacc.alloc(field_bytes(f)));
    if (m->ot == 4)
        for (int i = 0; i < 3; ++i) CK_TRY(m->z4[i].alloc(field_bytes(f)));   // halos stay zero
    CK_TRY(m->flags.alloc(sizeof(int) * 8));
    CK_TRY(m->phi.alloc(sizeof(double) * 2));
    CK_TRY(m->partials.alloc(sizeof(double) * m->nparts));
    *out = guard.release();
    return CKFWI_OK;
}

int ckfwi_set_model(ckfwi_model* m, const float* data, int kind, int mem, void* stream)
{
    if (!m || !data || (kind != CKFWI_VELOCITY && kind != CKFWI_SLOWNESS2)) return CKFWI_EINVAL;
    cudaStream_t st = S(stream);
    const FieldGeom& f = m->fg;
    DevMem tmp;
    const float* src = data;
    if (mem == CKFWI_HOST) {
        CK_TRY(tmp.alloc((size_t)f.npts * sizeof(float), false));
        CK_TRY(cudaMemcpyAsync(tmp.p, data, (size_t)f.npts * sizeof(float), cudaMemcpyHostToDevice, st));
        src = tmp.as<float>();
    }
    ST_TRY(reset_flags(m, st));
    ++m->model_ver;
    m->have_model = false;
    CK_TRY(launch_to_padded_w(src, kind, (float)m->g.dt, f, org(m->w, f), m->cvel.as<float>(),
                              m->flags.as<int>() + 2, st));
    int h[4];
    CK_TRY(cudaMemcpyAsync(h, m->flags.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK_TRY(cudaStreamSynchronize(st));
    if (h[2] & 2) return CKFWI_NONFINITE;
    if (h[2] & 1) return CKFWI_EINVAL;
    m->have_model = true;
    return CKFWI_OK;
}

int ckfwi_forward_shot(ckfwi_model* m, const ckfwi_shot* s, float* d_sim, int mem, void* stream)
{
    if (!m || !d_sim) return CKFWI_EINVAL;
    if (!m->have_model) return CKFWI_EINVAL;
    cudaStream_t st = S(stream);
    ST_TRY(set_shot(m, s));
    ST_TRY(autotune(m, st));
    ST_TRY(reset_flags(m, st));
    Ctx cx{m, st, 0};
    CK_TRY(cudaMemsetAsync(m->shot.dsim.p, 0, m->shot.dsim.bytes, st));
    State sv{ZERO_R, ZERO_R, U_FP32, U_FP32};
    for (int n = 0; n < m->g.nt; ++n) {
        const Role out = pick_free(sv);
        ST_TRY(fwd_step(cx, sv.cur, sv.prev, out, n, true, CK_NONE, NONE_R, NONE_R));
        sv.prev = sv.cur;
        sv.cur = out;
    }
    ST_TRY(sample_last(cx, sv.cur));
    const size_t nd = (size_t)(m->g.nt + 1) * m->shot.nrec;
    CK_TRY(cudaMemcpyAsync(d_sim, m->shot.dsim.p, nd * sizeof(float),
                           mem == CKFWI_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    // the kernels' error flags (a bounded wait that ran out); synchronises
    int fl = 0;
    ST_TRY(read_flags(m, st, &fl));
    return fl;
}

int ckfwi_misfit(ckfwi_model* m, const ckfwi_shot* s, const float* d_obs, int mem, double* misfit, float* d_sim,
                 void* stream)
{
    if (!m || !d_obs || !misfit || !m->have_model) return CKFWI_EINVAL;
    cudaStream_t st = S(stream);
    ST_TRY(set_shot(m, s));
    ST_TRY(autotune(m, st));
    ST_TRY(reset_flags(m, st));
    Ctx cx{m, st, 0};
    const size_t nd = (size_t)(m->g.nt + 1) * m->shot.nrec;
    CK_TRY(cudaMemcpyAsync(m->shot.dobs.p, d_obs, nd * sizeof(float),
                           mem == CKFWI_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    CK_TRY(cudaMemsetAsync(m->shot.dsim.p, 0, m->shot.dsim.bytes, st));
    State sv{ZERO_R, ZERO_R, U_FP32, U_FP32};
    for (int n = 0; n < m->g.nt; ++n) {
        const Role out = pick_free(sv);
        ST_TRY(fwd_step(cx, sv.cur, sv.prev, out, n, true, CK_NONE, NONE_R, NONE_R));
        sv.prev = sv.cur;
        sv.cur = out;
    }
    ST_TRY(sample_last(cx, sv.cur));
    ST_TRY(residual(cx));
    if (d_sim)
        CK_TRY(cudaMemcpyAsync(d_sim, m->shot.dsim.p, nd * sizeof(float),
                               mem == CKFWI_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    double phi = 0.0;
    CK_TRY(cudaMemcpyAsync(&phi, m->phi.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    int fl = 0;
    ST_TRY(read_flags(m, st, &fl));
    *misfit = phi;
    return fl;
}

int ckfwi_adjoint_gradient(ckfwi_model* m, const ckfwi_shot* s, const float* d_obs, int mem,
                           const ckfwi_grad_opts* opts, double* misfit, float* grad, ckfwi_stats* stats,
                           void* stream)
{
    if (!m || !grad) return CKFWI_EINVAL;
    cudaStream_t st = S(stream);
    const int rs = gradient_one(m, s, d_obs, mem, opts, misfit, stats, st);
    if (rs != CKFWI_OK) return rs;
    const FieldGeom& f = m->fg;
    const float scale = opts->grad_scale != 0.0 ? (float)opts->grad_scale : 1.0f;
    if (mem == CKFWI_HOST) {
        DevMem& tmp = m->hostgrad;     // kept: a host-buffer caller calls again with the same size
        CK_TRY(tmp.alloc((size_t)f.npts * sizeof(float), false));
        CK_TRY(launch_grad_out(org(m->gacc, f), m->cvel.as<float>(), opts->grad_kind, scale, f, tmp.as<float>(), st));
        CK_TRY(cudaMemcpyAsync(grad, tmp.p, (size_t)f.npts * sizeof(float), cudaMemcpyDeviceToHost, st));
        CK_TRY(cudaStreamSynchronize(st));
    } else {
        CK_TRY(launch_grad_out(org(m->gacc, f), m->cvel.as<float>(), opts->grad_kind, scale, f, grad, st));
        CK_TRY(cudaStreamSynchronize(st));
    }
    if (stats) stats->kernel_launches += 1;
    return CKFWI_OK;
}

int ckfwi_batch_gradient(ckfwi_model* m, const ckfwi_shot* shots, int nshots, const float* const* d_obs,
                         int mem, const ckfwi_grad_opts* opts, double* misfit_sum, double* grad_sum,
                         ckfwi_stats* stats, void* stream)
{
    if (!m || !shots || nshots < 1 || !d_obs || !grad_sum || !opts) return CKFWI_EINVAL;
    if (!m->have_model) return CKFWI_EINVAL;
    ST_TRY(check_opts(opts));
    cudaStream_t st = S(stream);
    const FieldGeom& f = m->fg;
    DevMem sum, comp;
    CK_TRY(sum.alloc((size_t)f.npts * sizeof(double)));
    CK_TRY(comp.alloc((size_t)f.npts * sizeof(double)));
    int B = batch_width(m, nshots, opts);
    double ms = 0.0, mc = 0.0;
    ckfwi_stats acc{};
    std::vector<double> phis((size_t)nshots, 0.0);
    for (int g0 = 0; g0 < nshots;) {
        const int nb = std::min(B, nshots - g0);
        ckfwi_stats one{};
        int rs = CKFWI_OK;
        std::vector<ckfwi_model*> lanes{m};
        if (nb == 1) {
            rs = gradient_one(m, shots + g0, d_obs[g0], mem, opts, &phis[g0], &one, st);
        } else {
            rs = ensure_clones(m, nb - 1, st);
            for (int l = 1; l < nb && rs == CKFWI_OK; ++l) lanes.push_back(m->clones[l - 1].get());
            if (rs == CKFWI_OK) rs = gradient_batch(lanes, shots + g0, d_obs + g0, mem, opts, &phis[g0], &one, st);
        }
        if (rs == CKFWI_ENOMEM && nb > 1) {
            // narrower batches, releasing the lanes that no longer fit
            B = std::max(1, nb / 2);
            m->clones.resize((size_t)(B - 1));
            CK_TRY(cudaDeviceSynchronize());
            continue;
        }
        ST_TRY(rs);
        // per-shot gradients into the FP64 sum, in shot order
        for (int l = 0; l < nb; ++l) {
            ckfwi_model* L = lanes[l];
            CK_TRY(launch_grad_out_f64(org(L->gacc, f), L->cvel.as<float>(), opts->grad_kind, f, 0, f.nx,
                                       (long long)f.ny * f.nx, sum.as<double>(), comp.as<double>(), st));
            const double phi = phis[g0 + l];
            const double t = ms + phi;
            mc += (std::fabs(ms) >= std::fabs(phi)) ? (ms - t) + phi : (phi - t) + ms;
            ms = t;
        }
        acc.fwd_steps += one.fwd_steps * nb;
        acc.adj_steps += one.adj_steps * nb;
        acc.p += one.p * nb;
        acc.takeshots += one.takeshots * nb;
        acc.restores += one.restores * nb;
        acc.kernel_launches += one.kernel_launches + nb;
        acc.fwd_launches += one.fwd_launches;
        acc.adj_launches += one.adj_launches;
        acc.comp_calls += one.comp_calls;
        acc.decomp_calls += one.decomp_calls;
        acc.fwd_ms += one.fwd_ms;
        acc.adj_ms += one.adj_ms;
        acc.comp_ms += one.comp_ms;
        acc.decomp_ms += one.decomp_ms;
        acc.other_ms += one.other_ms;
        acc.pool_bytes_peak = std::max(acc.pool_bytes_peak, one.pool_bytes_peak * nb);
        acc.u_absmax = std::max(acc.u_absmax, one.u_absmax);
        acc.fwd_ver = one.fwd_ver;
        acc.fwd_bx = one.fwd_bx;
        acc.fwd_by = one.fwd_by;
        acc.fwd_vec = one.fwd_vec;
        acc.fwd_zlen = one.fwd_zlen;
        acc.adj_ver = one.adj_ver;
        acc.adj_bx = one.adj_bx;
        acc.adj_by = one.adj_by;
        acc.adj_vec = one.adj_vec;
        acc.adj_zlen = one.adj_zlen;
        acc.fwd_pf = one.fwd_pf;
        acc.adj_pf = one.adj_pf;
        g0 += nb;
    }
    // sum + compensation, scaled; FP64 or rounded once to FP32
    const double scale = opts->grad_scale != 0.0 ? opts->grad_scale : 1.0;
    CK_TRY(launch_add_f64(sum.as<double>(), comp.as<double>(), scale, comp.as<double>(), f.npts, st));
    if (opts->grad_f32) {
        CK_TRY(launch_f64_to_f32(comp.as<double>(), sum.as<float>(), f.npts, st));
        CK_TRY(cudaMemcpyAsync(grad_sum, sum.p, f.npts * sizeof(float),
                               mem == CKFWI_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    } else {
        CK_TRY(cudaMemcpyAsync(grad_sum, comp.p, f.npts * sizeof(double),
                               mem == CKFWI_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    }
    CK_TRY(cudaStreamSynchronize(st));
    if (misfit_sum) *misfit_sum = ms + mc;
    if (stats) {
        *stats = acc;
        stats->ratio_min = 0;
        stats->ratio_mean = 0;
    }
    return CKFWI_OK;
}

int ckfwi_batch_gradient_models(ckfwi_model* const* models, const ckfwi_shot* shots, int nshots,
                                const float* const* d_obs, int mem, const ckfwi_grad_opts* opts,
                                const int* offsets, const int* global_n, double* misfit_sum, double* grad_sum,
                                ckfwi_stats* stats, void* stream)
{
    if (!models || !shots || nshots < 1 || !d_obs || !opts || !offsets || !global_n || !grad_sum)
        return CKFWI_EINVAL;
    ST_TRY(check_opts(opts));
    cudaStream_t st = S(stream);
    std::vector<ckfwi_model*> lanes((size_t)nshots);
    std::set<ckfwi_model*> seen;
    for (int l = 0; l < nshots; ++l) {
        ckfwi_model* L = models[l];
        if (!L || !L->have_model || !seen.insert(L).second) return CKFWI_EINVAL;
        if (L->ot == 4 && nshots > 1) return CKFWI_EINVAL;   // OT4 has no batched kernels
        lanes[l] = L;
        const FieldGeom& f = L->fg;
        const int n3[3] = {f.nz, f.ny, f.nx};
        for (int a = 0; a < 3; ++a)
            if (offsets[3 * l + a] < 0 || global_n[a] < 1 || offsets[3 * l + a] + n3[a] > global_n[a])
                return CKFWI_EINVAL;
    }
    const long long gn = (long long)global_n[0] * global_n[1] * global_n[2];
    DevMem sum, comp;
    CK_TRY(sum.alloc((size_t)gn * sizeof(double)));
    CK_TRY(comp.alloc((size_t)gn * sizeof(double)));
    std::vector<double> phis((size_t)nshots, 0.0);
    ckfwi_stats one{};
    if (nshots == 1) ST_TRY(gradient_one(lanes[0], shots, d_obs[0], mem, opts, &phis[0], &one, st));
    else ST_TRY(gradient_batch(lanes, shots, d_obs, mem, opts, phis.data(), &one, st));
    double ms = 0.0, mc = 0.0;
    for (int l = 0; l < nshots; ++l) {
        ckfwi_model* L = lanes[l];
        const FieldGeom& f = L->fg;
        const long long o0 =
            ((long long)offsets[3 * l] * global_n[1] + offsets[3 * l + 1]) * global_n[2] + offsets[3 * l + 2];
        CK_TRY(launch_grad_out_f64(org(L->gacc, f), L->cvel.as<float>(), opts->grad_kind, f, o0, global_n[2],
                                   (long long)global_n[1] * global_n[2], sum.as<double>(), comp.as<double>(), st));
        const double phi = phis[l];
        const double t = ms + phi;
        mc += (std::fabs(ms) >= std::fabs(phi)) ? (ms - t) + phi : (phi - t) + ms;
        ms = t;
    }
    const double scale = opts->grad_scale != 0.0 ? opts->grad_scale : 1.0;
    CK_TRY(launch_add_f64(sum.as<double>(), comp.as<double>(), scale, comp.as<double>(), gn, st));
    if (opts->grad_f32) {
        CK_TRY(launch_f64_to_f32(comp.as<double>(), sum.as<float>(), gn, st));
        CK_TRY(cudaMemcpyAsync(grad_sum, sum.p, gn * sizeof(float),
                               mem == CKFWI_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    } else {
        CK_TRY(cudaMemcpyAsync(grad_sum, comp.p, gn * sizeof(double),
                               mem == CKFWI_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    }
    CK_TRY(cudaStreamSynchronize(st));
    if (misfit_sum) *misfit_sum = ms + mc;
    if (stats) {
        *stats = one;
        stats->fwd_steps *= nshots;
        stats->adj_steps *= nshots;
        stats->p *= nshots;
        stats->takeshots *= nshots;
        stats->restores *= nshots;
        stats->kernel_launches += nshots;
    }
    return CKFWI_OK;
}

void ckfwi_free(ckfwi_model* m) { delete m; }

int ckfwi_stream_words(const ckfwi_model* m, long long* words, long long cap, long long* n)
{
    if (!m || !n || cap < 0 || (cap > 0 && !words)) return CKFWI_EINVAL;
    *n = (long long)m->last_words.size();
    if (cap < *n) return cap == 0 ? CKFWI_OK : CKFWI_EINVAL;
    std::copy(m->last_words.begin(), m->last_words.end(), words);
    return CKFWI_OK;
}

const char* ckfwi_error_string(int status)
{
    switch (status) {
    case CKFWI_OK: return "ok";
    case CKFWI_EINVAL: return "invalid argument";
    case CKFWI_ENOMEM: return "out of memory";
    case CKFWI_POOL_OVERFLOW: return "compressed checkpoints exceeded the pool";
    case CKFWI_NONFINITE: return "non-finite value";
    case CKFWI_CORRUPT: return "corrupt compressed stream";
    case CKFWI_TIMEOUT: return "device wait timed out";
    case CKFWI_ECUDA: return "CUDA runtime error";
    default: return "unknown status";
    }
}

int ckfwi_revolve_schedule(int nt, int slots, int32_t* actions, long long cap, long long* n_triples,
                           long long* counts)
{
    return ckfwi_multistage_schedule(nt, slots, 0, actions, cap, n_triples, counts);
}

int ckfwi_multistage_schedule(int nt, int slots, int host_slots, int32_t* actions, long long cap,
                              long long* n_triples, long long* counts)
{
    if (nt < 1 || slots < 1 || host_slots < 0 || host_slots > slots - 1) return CKFWI_EINVAL;
    std::vector<Action> acts;
    long long cnt[3];
    const int rc = host_slots > 0 ? multistage_schedule(nt, slots, host_slots, acts, cnt)
                                  : revolve_schedule(nt, slots, acts, cnt);
    if (rc != 0) return CKFWI_EINVAL;
    if (n_triples) *n_triples = (long long)acts.size();
    if (counts) {
        counts[0] = cnt[0];
        counts[1] = cnt[1];
        counts[2] = cnt[2];
    }
    if (!actions) return cap == 0 ? CKFWI_OK : CKFWI_EINVAL;
    if ((long long)acts.size() > cap) return CKFWI_EINVAL;
    for (size_t i = 0; i < acts.size(); ++i) {
        actions[3 * i] = acts[i].op;
        actions[3 * i + 1] = acts[i].a;
        actions[3 * i + 2] = acts[i].b;
    }
    return CKFWI_OK;
}

long long ckfwi_codec_bound_words(int dims, int nz, int ny, int nx)
{
    if ((dims != 2 && dims != 3) || nz < 1 || ny < 1 || nx < 1 || (dims == 2 && ny != 1)) return CKFWI_EINVAL;
    return codec_bound_words(dims, nz, ny, nx);
}

}  // extern "C"

namespace {
std::mutex g_codec_mu;
DevMem* g_codec_scratch[64] = {};
DevMem* g_codec_scal[64] = {};
}  // namespace

extern "C" int ckfwi_codec_compress(const float* x, int dims, int nz, int ny, int nx, double tol, uint32_t* out,
                                    long long cap, long long* used_words, int* flags, void* stream)
{
    if (!x || !out || cap <= 0) return CKFWI_EINVAL;
    if ((dims != 2 && dims != 3) || nz < 1 || ny < 1 || nx < 1 || (dims == 2 && ny != 1)) return CKFWI_EINVAL;
    if (!(tol >= std::ldexp(1.0, -90)) || !std::isfinite(tol)) return CKFWI_EINVAL;
    cudaStream_t st = S(stream);
    int dev = 0;
    CK_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return CKFWI_EINVAL;
    std::lock_guard<std::mutex> lk(g_codec_mu);
    if (!g_codec_scratch[dev]) g_codec_scratch[dev] = new DevMem();
    if (!g_codec_scal[dev]) g_codec_scal[dev] = new DevMem();
    DevMem& scr = *g_codec_scratch[dev];
    DevMem& scal = *g_codec_scal[dev];
    const size_t need = (size_t)codec_scratch_bytes(dims, nz, ny, nx);
    if (scr.bytes < need) CK_TRY(scr.alloc(need, false));
    CK_TRY(scal.alloc(64, true));
    CK_TRY(cudaMemsetAsync(scal.p, 0, 64, st));
    // the scratch serves fields of any size here: its counter and group sums
    // are cleared for this one's layout
    CK_TRY(cudaMemsetAsync(scr.p, 0, (size_t)codec_scratch_zero_bytes(dims, nz, ny, nx), st));
    CodecView v{};
    v.dims = dims; v.nz = nz; v.ny = ny; v.nx = nx;
    v.py = nx;
    v.pz = (long long)ny * nx;
    v.aligned = (nx % 4 == 0) && ((reinterpret_cast<uintptr_t>(x) & 15) == 0);
    long long* sc = scal.as<long long>();
    int* err = reinterpret_cast<int*>(sc + 4);
    CK_TRY(codec_compress_dev(x, v, tol_float(tol), out, sc, cap, sc + 1, scr.p, err, nullptr, st));
    long long h[5];
    CK_TRY(cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK_TRY(cudaStreamSynchronize(st));
    const int e = (int)(h[4] & 0xffffffff);
    if (flags) *flags = (e & 1) ? 1 : 0;
    if (e & 2) return CKFWI_POOL_OVERFLOW;
    if (e & 4) return CKFWI_CORRUPT;          // a chunk the compaction refused: the stream is incomplete
    if (used_words) *used_words = h[1];
    return CKFWI_OK;
}

extern "C" long long ckfwi_codec_rate_words(int dims, int nz, int ny, int nx, int rate)
{
    if ((dims != 2 && dims != 3) || nz < 1 || ny < 1 || nx < 1 || (dims == 2 && ny != 1)) return CKFWI_EINVAL;
    if (rate < 1 || rate > 32) return CKFWI_EINVAL;
    return codec_rate_words(dims, nz, ny, nx, rate);
}

extern "C" int ckfwi_codec_compress_rate(const float* x, int dims, int nz, int ny, int nx, int rate, uint32_t* out,
                                         long long cap, long long* used_words, int* flags, void* stream)
{
    if (!x || !out || cap <= 0) return CKFWI_EINVAL;
    if ((dims != 2 && dims != 3) || nz < 1 || ny < 1 || nx < 1 || (dims == 2 && ny != 1)) return CKFWI_EINVAL;
    if (rate < 1 || rate > 32) return CKFWI_EINVAL;
    cudaStream_t st = S(stream);
    int dev = 0;
    CK_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return CKFWI_EINVAL;
    std::lock_guard<std::mutex> lk(g_codec_mu);
    if (!g_codec_scal[dev]) g_codec_scal[dev] = new DevMem();
    DevMem& scal = *g_codec_scal[dev];
    CK_TRY(scal.alloc(64, true));
    CK_TRY(cudaMemsetAsync(scal.p, 0, 64, st));
    CodecView v{};
    v.dims = dims; v.nz = nz; v.ny = ny; v.nx = nx;
    v.py = nx;
    v.pz = (long long)ny * nx;
    v.aligned = false;
    long long* sc = scal.as<long long>();
    int* err = reinterpret_cast<int*>(sc + 4);
    CK_TRY(codec_rate_compress_dev(x, v, rate, out, sc, cap, sc + 1, err, nullptr, st));
    long long h[5];
    CK_TRY(cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK_TRY(cudaStreamSynchronize(st));
    const int e = (int)(h[4] & 0xffffffff);
    if (flags) *flags = (e & 1) ? 1 : 0;
    if (e & 2) return CKFWI_POOL_OVERFLOW;
    if (used_words) *used_words = h[1];
    return CKFWI_OK;
}

extern "C" int ckfwi_codec_decompress(const uint32_t* in, long long nwords, int dims, int nz, int ny, int nx,
                                      float* x, void* stream)
{
    if (!in || !x || nwords <= 0) return CKFWI_EINVAL;
    if ((dims != 2 && dims != 3) || nz < 1 || ny < 1 || nx < 1 || (dims == 2 && ny != 1)) return CKFWI_EINVAL;
    cudaStream_t st = S(stream);
    int dev = 0;
    CK_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return CKFWI_EINVAL;
    std::lock_guard<std::mutex> lk(g_codec_mu);
    if (!g_codec_scal[dev]) g_codec_scal[dev] = new DevMem();
    DevMem& scal = *g_codec_scal[dev];
    CK_TRY(scal.alloc(64, true));
    CK_TRY(cudaMemsetAsync(scal.p, 0, 64, st));
    CodecView v{};
    v.dims = dims; v.nz = nz; v.ny = ny; v.nx = nx;
    v.py = nx;
    v.pz = (long long)ny * nx;
    v.aligned = (nx % 4 == 0) && ((reinterpret_cast<uintptr_t>(x) & 15) == 0);
    long long* sc = scal.as<long long>();
    int* err = reinterpret_cast<int*>(sc + 4);
    // the header's version word says which mode wrote the stream
    uint32_t hv[9] = {};
    if (nwords < 16) return CKFWI_CORRUPT;
    CK_TRY(cudaMemcpyAsync(hv, in, sizeof(hv), cudaMemcpyDeviceToHost, st));
    CK_TRY(cudaStreamSynchronize(st));
    if ((hv[1] >> 8) == 2u) {
        if (hv[8] < 1u || hv[8] > 32u) return CKFWI_CORRUPT;   // the rate word of a fixed-rate stream
        CK_TRY(codec_rate_decompress_dev(in, sc, nwords, v, (int)hv[8], x, err, st));
    } else {
        CK_TRY(codec_decompress_dev(in, sc, nwords, v, x, err, st));
    }
    int e = 0;
    CK_TRY(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK_TRY(cudaStreamSynchronize(st));
    if (e & 4) return CKFWI_CORRUPT;
    return CKFWI_OK;
}
