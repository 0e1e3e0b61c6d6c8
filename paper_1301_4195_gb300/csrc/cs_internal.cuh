// Internal declarations shared by the CUDA translation units of libcs.
//
// Device data layouts (all in HBM, owned by the handle unless noted):
//   state f, Q, Qt       [ncells][N^3] double            (caller's layout, include/cs.h)
//   spectral F, Qhat     [ngroups][N^3][32] complex T     (T = double or float)
//                        cells in groups of 32, one cell per warp lane, so a
//                        warp reads 32 consecutive complex values per grid point
//   weight table         [pencil (k1,k2)][tile][pair] T, see weights.cu
//   transform scratch    [ncells][N^3] complex T (two buffers)
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cs.h"

namespace cs {

constexpr int kGroup = 32;  // cells per group (= warp lanes)
constexpr int kMaxN = 64;
constexpr int kMaxLeg = 16;  // Legendre moments of an anisotropic b(cos theta)

template <typename T> struct C2;
template <> struct C2<double> { using type = double2; };
template <> struct C2<float> { using type = float2; };
template <typename T> using c2_t = typename C2<T>::type;

// Order of the (m3, k3) pairs inside one weight tile.
//   ROWS:  rows m3 = 0..N-1, each row the valid k3 ascending, padded to a
//          multiple of 4 entries (generic and pencil kernels).
//   STRIP: for the strip kernel (float, N in {8, 16, 24, 32, 48, 64}): the k3 range is
//          cut into strips of K outputs; each strip's pairs are stored together
//          (see strip_* below).
enum Layout { LAYOUT_ROWS = 0, LAYOUT_STRIP = 1 };

// Geometry of one handle, passed to kernels by value.
struct Geom {
    int N, h, M;          // h = N/2, M = N^3
    int TS, TSp;          // valid (m3,k3) pairs per tile = 3N^2/4; tile stride of the layout
    int layout, K;        // tile layout and, for LAYOUT_STRIP, the strip width
    double L, dv, dz;     // half-width, velocity and Fourier spacings
    double lambda;
    int off[kMaxN + 1];   // ROWS layout: off[m3] = first entry of row m3 inside a tile
    // anisotropic scattering: b(cos theta) by its Legendre moments
    // bl[l] = int_{S^2} b(t) P_l(t) dsigma, l < nleg (nleg = 0: isotropic 1/4pi)
    int nleg;
    double bl[kMaxLeg];
};

__host__ __device__ inline int kmin_of(int m3, int h) { return m3 - h > 0 ? m3 - h : 0; }
__host__ __device__ inline int kmax_of(int m3, int h, int N) { return m3 + h - 1 < N - 1 ? m3 + h - 1 : N - 1; }

// ---- STRIP layout.  Strip w covers k3 in [k0, k0 + K), k0 = w K, K | N/2,
// K % 4 == 0.  With H = N/2 a strip is of one of two kinds:
//   A (k0 < H):  "uniform" rows m3 = 0 .. k0 + H (all K outputs valid, K entries
//                each), then a triangle t = 1 .. K-1: m3 = k0 + H + t with
//                outputs j = t .. K-1 (K - t entries each);
//   B (k0 >= H): triangle t = 0 .. K-2: m3 = k0 - H + 1 + t with outputs
//                j = 0 .. t, padded to a multiple of 4 entries, then uniform
//                rows m3 = k0 + K - H .. N - 1.
// Strips are stored one after another, each padded to a multiple of 4.
__host__ __device__ constexpr int strip_round4(int x) { return (x + 3) & ~3; }
__host__ __device__ constexpr bool strip_is_a(int N, int K, int w) { return w * K < N / 2; }
__host__ __device__ constexpr int strip_lu(int N, int K, int w)
{
    return strip_is_a(N, K, w) ? w * K + N / 2 + 1 : N + N / 2 - w * K - K;
}
__host__ __device__ constexpr int strip_tri(int K) { return K * (K - 1) / 2; }
__host__ __device__ constexpr int strip_seg_size(int N, int K, int w) { return strip_lu(N, K, w) * K + strip_round4(strip_tri(K)); }
__host__ __device__ constexpr int strip_seg_off(int N, int K, int w)
{
    int o = 0;
    for (int i = 0; i < w; ++i) o += strip_seg_size(N, K, i);
    return o;
}
__host__ __device__ constexpr int strip_stride(int N, int K) { return strip_seg_off(N, K, N / K); }
__host__ __device__ constexpr int strip_tri_a_off(int K, int t)  // kind A, rows t = 1 .. K-1
{
    int o = 0;
    for (int i = 1; i < t; ++i) o += K - i;
    return o;
}
__host__ __device__ constexpr int strip_tri_b_off(int t) { return t * (t + 1) / 2; }  // kind B, rows t = 0 .. K-2

// strip width used for (N, float); 0 = the strip kernel does not serve N
__host__ __device__ constexpr int strip_width(int N)
{
    return N == 8 ? 4 : N == 16 ? 8 : N == 24 ? 12 : (N == 32 || N == 48 || N == 64) ? 8 : 0;
}

struct Handle {
    int device = 0;
    int precision = CS_FP64;
    Geom g{};
    // weights
    void *ghat = nullptr;         // T[total_tiles * TSp]
    size_t ghat_bytes = 0;
    long long total_tiles = 0;
    int *pencil_tile0 = nullptr;  // device int[N*N + 1]: first tile of each pencil
    int *pencil_order = nullptr;  // device int[N*N]: pencils by decreasing tile count
    std::vector<int> order_host;
    // radius tables (float strip handles): A[|k'|^2][|2m'-k'|^2], B[|m'|^2], and
    // the tile entry map; the strip kernel rebuilds weight tiles from them
    float *radA = nullptr, *radB = nullptr;
    int *emap = nullptr;
    int rad_bb = 0;               // row length of A
    size_t rad_bytes = 0;
    bool has_table = true;        // false: built with CS_WEIGHTS_RADIUS (no stored tiles)
    int *err = nullptr;           // device word: bit 0 set when a bounded device wait expired
    int *counter = nullptr;       // device word: work counter of the persistent convolution (err + 32)
    // transforms: twiddles exp(-i 2 pi ((k-h)(j-h) mod N) / N), [k][j]
    double2 *tw64 = nullptr;
    float2 *tw32 = nullptr;
    // projection
    double cct_inv[25] = {};
    // workspace
    int ws_cells = 0;
    int ws_geo_cells = 0;         // grid size the transport tables have room for
    // what the transport tables in `scal` were last prepared for by
    // cs_transport_shard_prepare (total_cells < 0: not prepared, or
    // overwritten since by cs_transport / cs_step or a workspace move)
    struct {
        int total_cells = -1;
        const double *dx = nullptr;
        double wall_T = 0, wall_V[3] = {0, 0, 0};
    } shard_tables;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    unsigned ws_generation = 0;  // bumped whenever the workspace moves
    // pieces of the workspace (set by layout_workspace)
    void *F = nullptr, *Qh = nullptr, *X = nullptr, *Y = nullptr;
    void *Fc = nullptr;  // the few-cell kernel's f-hat of up to 16 cells (conv_lane.cu), or none
    // partial sums 2-4 of a split convolution (conv_split > 1; the kernel's
    // last part adds them into Qh): Qh2 aliases X, Qh3 aliases Y (scratch of
    // the per-axis transforms, which split handles do not use), Qh4 and the
    // per-(pencil, block) counters of finished parts have room of their own
    void *Qh2 = nullptr, *Qh3 = nullptr, *Qh4 = nullptr;
    int *done = nullptr;
    double *Qt = nullptr, *f1 = nullptr, *r1 = nullptr, *scal = nullptr;
    double *part5 = nullptr;  // per-block partial moments of the projection
    // replayable steps (cs_step, cs_relax): one captured step per argument set
    struct GraphEntry {
        int kind;  // 1 = Strang step, 2 = homogeneous Heun step, 3 = Strang step in 2-D, 4 = in 3-D
        const void *f, *dx, *ffar;
        int ncells;
        double wall_T, wall_V[3], dt, eps;
        cudaGraphExec_t exec;
        int kernels;  // kernel nodes of the captured step
        int ny;       // 2-D, 3-D: cells across y, and their width
        double dy;
        int nz;       // 3-D: cells across z, and their width
        double dz;
    };
    std::vector<GraphEntry> graphs;
    cudaStream_t cap_stream = nullptr;
    bool use_graphs = true;
    // convolution launch choices (0 = automatic), set by cs_tune / cs_autotune
    int tune_gpc = 0;     // cell groups per CTA of the strip kernel (1 or 2)
    int tune_ctas = 0;    // resident CTAs per SM of the persistent strip kernel
    int tune_weights = 0; // 1 = stored tiles, 2 = tiles rebuilt from the radius tables
    int tune_split = 0;   // tile ranges per pencil at N = 16 (2 or 4; 0 = 2)
    int tune_l2 = 0;      // L2 eviction priorities on the convolution's copies (1 off, 2 on; 0 = on)
    int tune_tile = 0;    // xi-tile and ring depth (1 = U 8 with 3 stages, the default; 2 .. 4 see conv_tiles.cu)
    int tune_few = 0;     // most cells the few-cell kernel serves (0 = its default, -1 = never; conv_lane.cu)
    // checks (cs_tune): limit of the convolution's bounded waits (us, 0 =
    // 2 s), the stall that makes them run out in tests, the input scan
    // (0 off, 1 non-finite, 2 non-finite or negative), and whether a Heun
    // step's first inverse launch also transforms forward (2 = no)
    unsigned wait_us = 0;
    int test_stall = 0;
    int check_input = 0;
    int tune_fwd_next = 0;
    // stage timing (cs_profile)
    bool prof = false;
    struct Rec {
        cudaEvent_t a, b;
        int k;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
};

// Brackets one stage with events when profiling is on (cs_api.cu).
class StageTimer {
public:
    StageTimer(Handle &hd, int k, cudaStream_t s);
    ~StageTimer();

private:
    Handle *hd_;
    cudaStream_t s_;
    int k_;
    cudaEvent_t b_ = nullptr;
};

// ---- errors (cs_api.cu)
int set_error(int code, const std::string &msg);
int cuda_error(cudaError_t e, const char *what);
#define CS_CHECK_LAUNCH(what)                                    \
    do {                                                         \
        cudaError_t _e = cudaGetLastError();                     \
        if (_e != cudaSuccess) return ::cs::cuda_error(_e, what); \
    } while (0)
// Library-wide count of kernels put on streams (cs_launch_count): n launches
// just enqueued on s count now unless s is being captured, in which case the
// graph's kernel nodes count at each replay instead.
void note_kernels(cudaStream_t s, int n);
int graph_kernel_nodes(cudaGraph_t g);
void note_replay(int kernels);
#define CS_LAUNCHED(n, s, what)        \
    do {                               \
        CS_CHECK_LAUNCH(what);         \
        ::cs::note_kernels((s), (n));  \
    } while (0)

inline size_t elem_bytes(int precision) { return precision == CS_FP32 ? 4 : 8; }
inline int ngroups_of(int ncells) { return (ncells + kGroup - 1) / kGroup; }

// ---- cs_api.cu
void fill_geom(Geom &g, int N, double L, double lambda, int precision);
// entry map of one tile: map[p] = (m3 << 8) | k3, or -1 for padding; size g.TSp
void tile_entry_map(const Geom &g, std::vector<int> &map);

// ---- weights.cu
long long count_tiles(int N, int *pencil_tile0_host /* may be null, size N*N+1 */);
int build_weights(Handle &hd, cudaStream_t s);
// radius tables of a float strip handle: dimensions, bytes (0 where the strip
// kernel does not serve N), build
void radius_dims(int N, int *KK, int *BB, int *MM);
size_t radius_bytes(int N);
int build_radius_tables(Handle &hd, cudaStream_t s);
int sample_weights(Handle &hd, const int *km_host, int n, double *out_host);

// ---- transform.cu
int launch_forward(const Handle &hd, const double *f, int ncells, cudaStream_t s);   // f -> hd.F
// hd.Qh -> Qt
int launch_inverse(const Handle &hd, int ncells, double scale_eps, double *Qt, cudaStream_t s);
// grouped spectral src -> [ncells][N^3][2] doubles
int launch_spectral_to_natural(const Handle &hd, const void *src, int ncells, double *dst, cudaStream_t s);
int launch_natural_to_spectral(const Handle &hd, const double *src, int ncells, void *dst, cudaStream_t s);

// ---- fused.cu (float, N <= 24: whole-cell transforms in shared memory)
bool fused_available(const Handle &hd);
// fhat of cells 0 .. ncells-1, zeros for the cells up to max(ncells, grid_cells)
// rounded up to whole 32-cell groups
int launch_forward_fused(const Handle &hd, const double *f, int ncells, cudaStream_t s, int grid_cells = 0);
// out = a x + b y + P(c Qt), Qt the inverse transform of hd.Qh (+ qh2 if not
// NULL), P the projection if project (else the identity)
// With fnext (not NULL; only where fused_forward_next) the same launch then
// transforms `out` forward into fnext, in the grouped layout the convolution
// reads: the forward transform of a Heun step's second evaluation.
int launch_inverse_project(const Handle &hd, int ncells, double eps, int project, double a, const double *x,
                           double b, const double *y, double c, double *out, cudaStream_t s,
                           void *fnext = nullptr);
bool fused_forward_next(const Handle &hd);  // one block per cell: float, N in {8, 12, 16, 24}

// ---- convolve.cu, conv_strip.cu
int launch_convolve(const Handle &hd, int ncells, cudaStream_t s);  // hd.F -> hd.Qh (and hd.Qh2)
// into how many tile ranges the convolution of this handle splits each
// pencil: 2 or 4 for float strip handles at N = 16 (CS_TUNE_SPLIT, default
// 2), else 1; the last range to finish adds the partial sums into hd.Qh in
// range order, so every consumer reads one buffer.  The split fixes the
// summation order, so it is a property of the handle, never of a call.
int conv_split(const Handle &hd);
int conv_split_max(const Handle &hd);  // the largest split the handle's workspace must hold
int launch_strip(const Handle &hd, int ncells, cudaStream_t s);     // float, LAYOUT_STRIP
int launch_strip_radius(const Handle &hd, int ncells, cudaStream_t s);  // conv_radius.cu
// conv_tiles.cu: the strip launch with the tile shape hd.tune_tile (2: U = 4;
// 3: a 4-stage ring; 4: a 2-stage ring) at N = 16 and 32, stored tiles
int launch_strip_tiles(const Handle &hd, int ncells, cudaStream_t s);
int launch_strip_split32(const Handle &hd, int ncells, cudaStream_t s, bool rad);  // conv_split32.cu: N = 32, S = 2, 4
bool lane_conv_capable(const Handle &hd);                           // conv_lane.cu: the handle's kind has a few-cell kernel
bool lane_conv_applies(const Handle &hd, int ncells);               // conv_lane.cu: the few-cell kernel serves the call
int launch_strip_lane(const Handle &hd, int ncells, cudaStream_t s);  // its transpose and convolution launches
bool tile_shapes_available(const Handle &hd);
bool strip_uses_radius(const Handle &hd);  // the handle's strip launches rebuild tiles from the radius tables

// ---- conv_mixed.cu: the convolutions of several float strip handles in one launch
bool strip_mixable(const Handle &hd);              // float, LAYOUT_STRIP, N in {8, 16, 24, 32}
int strip_mixed_cells(const Handle &hd, int ncells);  // cells its workspace and forward transform must cover
int launch_strip_mixed(const Handle *const *hds, const int *ncells, int n, cudaStream_t s);

// ---- conserve.cu
// out = a*x + b*y + c*(P Qt)   (P = projection if project, else identity), per cell
// x, y may be null when a, b are 0.  out may alias Qt, x or y elementwise.
int launch_conserve(const Handle &hd, const double *Qt, int ncells, int project, double a,
                    const double *x, double b, const double *y, double c, double *out,
                    double *moments, cudaStream_t s);
int launch_moments(const Handle &hd, const double *f, int ncells, double *out, cudaStream_t s);
int conserve_parts(int M);  // blocks per cell of the projection
// the input scan of CS_TUNE_CHECK_INPUT: sets bit 1 of hd.err if one of the
// ncells * N^3 values of f is not finite, bit 2 if one is negative (mode 2);
// enqueues nothing when the handle's scan is off
int launch_input_check(const Handle &hd, const double *f, long long count, cudaStream_t s);

// ---- transport.cu
// doubles of workspace the transport tables need; tables are filled by
// launch_transport_prep once per call (geometry, wall Maxwellian flux)
// transport tables (geometry, wall Maxwellian) for a grid of total_cells cells
size_t transport_table_doubles(int N, int total_cells);
int launch_transport_prep(const Handle &hd, int total_cells, const cs_domain &dom, cudaStream_t s);
// a stage of the transport in two space dimensions: fin, out [nx][ny][N^3],
// x the wall direction of dom, y periodic with ny cells of width dy
int launch_transport_stage2d(const Handle &hd, const double *fin, int nx, int ny, double dy, const cs_domain &dom,
                             double a, const double *x, double b, const double *y, double c, double *out,
                             cudaStream_t s);
// a stage in three space dimensions: fin, out [nx][ny][nz][N^3], y and z
// periodic with ny, nz cells of widths dy, dz
int launch_transport_stage3d(const Handle &hd, const double *fin, int nx, int ny, int nz, double dy, double dz,
                             const cs_domain &dom, double a, const double *x, double b, const double *y, double c,
                             double *out, cudaStream_t s);
// one transport stage, out = a x + b y + c rhs(fin), rhs the finite-volume
// operator, for cells first .. first+ncells-1, read from fin with `ghost`
// leading ghost cells (0: fin holds exactly the cells; 2: a window); out must
// not overlap fin (it may alias x or y)
int launch_transport_stage(const Handle &hd, const double *fin, int ghost, int first, int ncells, int total_cells,
                           const cs_domain &dom, double a, const double *x, double b, const double *y, double c,
                           double *out, cudaStream_t s);

}  // namespace cs

// The opaque handle of the C ABI.
struct cs_handle_s {
    cs::Handle h;
};
