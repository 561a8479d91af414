// Internal declarations of the ckfwi library (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace ckfwi {

constexpr int MAXK = 8;          // half space order, space orders 2..16

// Padded field layout.  Every wavefield carries H zero cells beyond each
// face of the total grid in z (and y in 3D) and at least H in x; those
// cells are never written, so they act as the zero Dirichlet values the
// Laplacian reads outside the grid.  Pointers handed to kernels are
// "origin based": element (z, y, x) of the total grid sits at
// p[z * pxy + y * px + x].  The first interior column is 16-byte aligned.
struct FieldGeom {
    int dims;
    int nz, ny, nx;     // total grid
    int H;              // halo depth in z (and y in 3D)
    int X0;             // x offset of column 0 inside a row (multiple of 4, >= H)
    long long px;       // row pitch [floats], multiple of 32
    long long pxy;      // plane pitch [floats]
    long long origin;   // offset of element (0,0,0) from the allocation start
    long long alloc;    // floats per field allocation
    long long npts;     // nz * ny * nx
};

FieldGeom make_geom(int dims, int nz, int ny, int nx, int H);

// Point sources on the grid, gathered through a CSR map over a bounding box:
// at a grid point inside the box, value = sum_e wt[e] * series[col[e]] over
// e in rowptr[b] .. rowptr[b+1]-1, b the point's index inside the box.
// A deterministic gather (no atomics), so every launch rounds identically.
struct Inj {
    int on;
    int z0, z1, y0, y1, x0, x1;   // half-open box in total-grid indices
    const int* rowptr;
    const int* col;
    const float* wt;
    const float* series;          // this step's values (already offset)
};

// Receiver sampling d_r = sum_i wt[r][i] * u[idx[r][i]] (multilinear weights).
struct Sample {
    int n;                        // receivers, 0 = off
    int nst;                      // 4 (2D) or 8 (3D)
    const long long* idx;         // origin-based offsets [n][nst]
    const float* wt;              // [n][nst]
    float* out;                   // [n]
};

// Forward OT2 step: a u^{n+1} = 2u^n - b u^{n-1} + w (lap u^n + Q^T s^n).
struct FwdArgs {
    FieldGeom g;
    const float* u;       // u^n
    const float* up;      // u^{n-1}
    const float* w;       // dt^2 c^2
    float* out;           // u^{n+1}
    const float* eta;     // damping tables: eta_z[nz], eta_y[ny], eta_x[nx]
    float hdt;            // dt / 2
    float c[MAXK + 1];    // c[j] = c_j / h^2 (j >= 1); c[0] unused
    int zlen;             // z planes per CTA
    Inj src;
    Sample smp;
    void* ck_u;           // fused takeshot outputs (see CkMode)
    void* ck_up;
    int* err;             // error flags (bit 0: FP16 overflow, bit 3: a bounded wait ran out)
    long long wait_limit; // TMA kernels: back-off rounds of a plane's bounded wait (< 0: give up at once)
};

// Fused reverse step:
//   a lam^{j-1} = 2 lam^j - b lam^{j+1} + w (lap lam^j - P^T r^j)
//   gacc += lam^{j-1} * (lap u^{j-1} + Q^T s^{j-1})
struct AdjArgs {
    FieldGeom g;
    const float* l1;      // lam^j
    const float* l2;      // lam^{j+1}
    float* l0;            // lam^{j-1}
    const void* u;        // u^{j-1}, element type per template
    const float* w;
    float* gacc;
    const float* eta;
    float hdt;
    float c[MAXK + 1];
    int zlen;
    Inj adj;              // -P^T r^j  (weights carry the minus sign)
    Inj src;              // Q^T s^{j-1}
    int* err;             // error flags (bit 3: a bounded wait ran out)
    long long wait_limit; // TMA kernels: back-off rounds of a plane's bounded wait (< 0: give up at once)
};

// OT4 kernel (Sec. 6): a forward step is two passes, Z = w lap f and then the
// leapfrog update with w A f = Z + w lap(Z) / 12; a reverse step is three
// (ot4.cu).
struct Ot4LapArgs {
    FieldGeom g;
    const float* f0;      // u^n (forward) or lam^j (reverse)
    const void* f1;       // reverse: u^{j-1}, element type per launch; forward: null
    float* z0;            // w lap f0
    float* z1;            // w lap f1
    const float* w;
    float c[MAXK + 1];
    int zlen;
    Sample smp;           // forward: receiver sampling of u^n
    float* gacc;          // reverse: gacc += zu_next lap(f0) / 12 (zu_next null: nothing)
    const float* zu_next; // reverse: w lap u^j from the previous reverse step
    float c12[MAXK + 1];  // c_j / (12 h^2)
};

struct Ot4FwdArgs {
    FwdArgs f;            // as OT2 (c unused); also the reverse update (u = lam^j, up = lam^{j+1})
    const float* z;       // w lap u^n (reverse: w lap lam^j)
    float c12[MAXK + 1];  // c_j / (12 h^2)
};

// The reverse step's gradient pass: gacc += lam^{j-1} (lap u^{j-1} + lap(Z_u)/12 + q^{j-1}).
struct Ot4GradArgs {
    FieldGeom g;
    const void* u;        // u^{j-1}, element type per launch
    const float* zu;      // w lap u^{j-1}
    const float* l0;      // lam^{j-1}
    float* gacc;
    float c[MAXK + 1];
    float c12[MAXK + 1];
    int zlen;
    Inj src;              // Q^T s^{j-1}
};

enum CkMode { CK_NONE = 0, CK_FP32 = 1, CK_BF16 = 2, CK_FP16 = 3 };
enum UType { U_FP32 = 0, U_BF16 = 1, U_FP16 = 2 };

struct Tile {
    int bx, by;           // CTA shape in points (by = 1 in 2D); TMA kernels: bx = 64 points, by rows
    int zlen;             // ver 1, 3: z planes per CTA; ver 2: CTAs per SM of the persistent grid
    int ver = 1;          // 1: register-queue kernels, 2: TMA-fed kernels (3D, orders 2-8),
                          // 3: vector-blocked kernels (3D), 4: vector-blocked forward step fed
                          // by asynchronous copies (3D), 5: the two-pass OT4 kernels,
                          // 6: the same vector-blocked (3D), 7: the lean async-copy
                          // OT2 kernels (3D, one or two planes per step), 8: the
                          // forward step fed by tensor copies and the reverse step split
                          // in two launches (3D)
    int vec = 1;          // ver 3, 4: x points per thread (2 or 4)
    int pf = 0;           // ver 4: planes of prefetch (0 = the default, 2); ver 7: planes per step (1, 2);
                          // ver 8: planes of prefetch (1, 2; 0 reads as 1)
};

// One batched step over several lanes (shots): lane l's arguments are
// tab[l] (device) and its CTAs start[l] .. start[l+1]-1 of a 1D grid of
// `blocks` CTAs (start: device, lanes + 1 entries).  Every lane's zlen is
// its own; the tile shape is common.
template <class Args>
struct BatchLaunch {
    const Args* tab;
    const int* start;
    int lanes;
    int dims;
    long long blocks;
};

// kernels.cu
cudaError_t launch_fwd(const FwdArgs& a, const Tile& t, int K, int ck, cudaStream_t s);
cudaError_t launch_fwd_batch(const BatchLaunch<FwdArgs>& b, const Tile& t, int K, int ck, cudaStream_t s);
cudaError_t launch_adj_batch(const BatchLaunch<AdjArgs>& b, const Tile& t, int K, int ut, cudaStream_t s);
cudaError_t launch_adj(const AdjArgs& a, const Tile& t, int K, int utype, cudaStream_t s);
bool tile_supported(int dims, int K, const Tile& t);
int tile_count(int dims);
Tile tile_at(int dims, int i, int zlen);

// stencil_v3.cu
int v3_shape_count();
Tile v3_tile_at(int i, int zlen);
bool v3_supported(int dims, int K, const Tile& t);
bool v3_fits(const FieldGeom& g, int K);
cudaError_t launch_fwd3(const FwdArgs& a, const Tile& t, int K, int ck, cudaStream_t s);
cudaError_t launch_adj3(const AdjArgs& a, const Tile& t, int K, int ut, cudaStream_t s);
// stencil_v4.cu (geometry must pass v3_fits)
bool v4_supported(int dims, int K, const Tile& t);
cudaError_t launch_fwd4(const FwdArgs& a, const Tile& t, int K, int ck, cudaStream_t s);
cudaError_t launch_adj4(const AdjArgs& a, const Tile& t, int K, int ut, cudaStream_t s);
// stencil_v5.cu: the lean async-copy generation (Tile.ver 7; geometry must pass v3_fits)
bool v5_supported(int dims, int K, const Tile& t);
cudaError_t launch_fwd5(const FwdArgs& a, const Tile& t, int K, int ck, cudaStream_t s);
cudaError_t launch_adj5(const AdjArgs& a, const Tile& t, int K, int ut, cudaStream_t s);
// batched forms of generations 4 and 7 (every lane's geometry must pass v3_fits)
cudaError_t launch_fwd4_batch(const BatchLaunch<FwdArgs>& b, const Tile& t, int K, int ck, cudaStream_t s);
cudaError_t launch_fwd5_batch(const BatchLaunch<FwdArgs>& b, const Tile& t, int K, int ck, cudaStream_t s);
cudaError_t launch_adj5_batch(const BatchLaunch<AdjArgs>& b, const Tile& t, int K, int ut, cudaStream_t s);
// batch_v3.cu (every lane's geometry must pass v3_fits)
cudaError_t launch_fwd3_batch(const BatchLaunch<FwdArgs>& b, const Tile& t, int K, int ck, cudaStream_t s);
cudaError_t launch_adj3_batch(const BatchLaunch<AdjArgs>& b, const Tile& t, int K, int ut, cudaStream_t s);

// ot4.cu
bool ot4_supported(int dims, int K, const Tile& t);
int ot4_shape_count(int dims);
Tile ot4_tile_at(int dims, int i, int zlen);
cudaError_t launch_ot4_lap(const Ot4LapArgs& a, const Tile& t, int K, int ut, cudaStream_t s);
cudaError_t launch_ot4_fwd(const Ot4FwdArgs& a, const Tile& t, int K, int ck, cudaStream_t s);
cudaError_t launch_ot4_grad(const Ot4GradArgs& a, const Tile& t, int K, int ut, cudaStream_t s);
// ot4_v3.cu: the same passes vector-blocked (3D, geometry must pass v3_fits)
bool ot4v_supported(int dims, int K, const Tile& t, bool reverse);
cudaError_t launch_ot4v_lap(const Ot4LapArgs& a, const Tile& t, int K, int ut, cudaStream_t s);
cudaError_t launch_ot4v_fwd(const Ot4FwdArgs& a, const Tile& t, int K, int ck, cudaStream_t s);
cudaError_t launch_ot4v_grad(const Ot4GradArgs& a, const Tile& t, int K, int ut, cudaStream_t s);

// stencil_tma.cu (CUtensorMap comes from <cuda.h>)
}  // namespace ckfwi
#include <cuda.h>
namespace ckfwi {
int tma_halo_x(int K);
int tma_tile_x();
bool tma_supported(int dims, int K, int ty);
cudaError_t launch_fwd_tma(const FwdArgs& a, const CUtensorMap& tmu, const Tile& t, int K, int ck, cudaStream_t s);
cudaError_t launch_adj_tma(const AdjArgs& a, const CUtensorMap& tml, const CUtensorMap& tmu, const Tile& t, int K,
                           int ut, cudaStream_t s);
// stencil_tq.cu: the forward step fed by tensor copies (Tile.ver 8; geometry
// must pass v3_fits; tu: box tq_box_x x tq_box_y of u, tp / tw: 32 x 16 of
// u^{n-1} / w, maps of the padded device allocations)
bool tq_supported(int dims, int K, const Tile& t);
int tq_box_x(int K);
int tq_box_y(int K);
cudaError_t launch_fwdq(const FwdArgs& a, const CUtensorMap& tu, const CUtensorMap& tp, const CUtensorMap& tw,
                        const Tile& t, int K, int ck, cudaStream_t s);
// the reverse step split in two launches: the lam half by fwdq_kernel (maps
// 0-2: lam^j with the u box, lam^{j+1} and w with point boxes), then the
// gradient half (maps 3-5: u^{j-1} with the u box, lam^{j-1} and g with
// point boxes); FP32 u^{j-1} only
cudaError_t launch_adjq(const AdjArgs& a, const CUtensorMap* maps, const Tile& t, int K, cudaStream_t s);

// aux.cu
cudaError_t launch_sample(const float* u, const Sample& smp, cudaStream_t s);
// *out = max(*out, bits of max |u|) over the total grid (out must start at 0)
cudaError_t launch_absmax(const float* u_origin, const FieldGeom& g, unsigned* out, cudaStream_t s);
cudaError_t launch_residual(const float* d, const float* dobs, float* r, int rows, int nrec,
                            double* partials, int nparts, double* phi, cudaStream_t s);
cudaError_t launch_to_padded_w(const float* dense, int kind, float dt, const FieldGeom& g,
                               float* w_origin, float* c2_dense, int* err, cudaStream_t s);
cudaError_t launch_grad_out(const float* gacc_origin, const float* c_dense, int kind, float scale,
                            const FieldGeom& g, float* out_dense, cudaStream_t s);
// Compensated FP64 sum of one shot's gradient into a dense array; grid
// point (z, y, x) adds at o0 + z * gsz + y * gsy + x.
cudaError_t launch_grad_out_f64(const float* gacc_origin, const float* c2_dense, int kind,
                                const FieldGeom& g, long long o0, long long gsy, long long gsz,
                                double* sum, double* comp, cudaStream_t s);
cudaError_t launch_cast_restore(const void* src, int utype, const FieldGeom& g,
                                float* dst_origin, cudaStream_t s);
cudaError_t launch_copy_f64(const double* a, double* b, long long n, cudaStream_t s);
cudaError_t launch_add_f64(const double* a, const double* b, double scale, double* out, long long n, cudaStream_t s);
cudaError_t launch_f64_to_f32(const double* a, float* out, long long n, cudaStream_t s);

// codec.cu
struct CodecView {       // a float field to (de)compress, origin based
    int dims, nz, ny, nx;
    long long py, pz;    // pitches [floats] of y rows and z planes
    bool aligned;        // rows 16-byte aligned with a multiple-of-4 pitch
};
long long codec_bound_words(int dims, int nz, int ny, int nx);
long long codec_scratch_bytes(int dims, int nz, int ny, int nx);
// leading bytes of that scratch that must be zero before a compression
// (a compression leaves them zero again)
long long codec_scratch_zero_bytes(int dims, int nz, int ny, int nx);
// Compress into `out` at word offset read from *base_word (device), checking
// against cap_words; writes *next_word = base + stream length (device) and
// raises err bits: 1 NONFINITE, 2 OVERFLOW.
cudaError_t codec_compress_dev(const float* x, const CodecView& v, float tol_f,
                               uint32_t* out, const long long* base_word, long long cap_words,
                               long long* next_word, void* scratch, int* err,
                               unsigned long long* stat_words, cudaStream_t s);
cudaError_t codec_decompress_dev(const uint32_t* in, const long long* base_word,
                                 long long cap_words, const CodecView& v, float* x, int* err,
                                 cudaStream_t s);
// codec_rate.cu: the fixed-rate mode (same pool conventions; rate 1..32)
long long codec_rate_words(int dims, int nz, int ny, int nx, int rate);
cudaError_t codec_rate_compress_dev(const float* x, const CodecView& v, int rate, uint32_t* out,
                                    const long long* base_word, long long cap_words, long long* next_word,
                                    int* err, unsigned long long* stat_words, cudaStream_t s);
cudaError_t codec_rate_decompress_dev(const uint32_t* in, const long long* base_word, long long cap_words,
                                      const CodecView& v, int rate, float* x, int* err, cudaStream_t s);

}  // namespace ckfwi
