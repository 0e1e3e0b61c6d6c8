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
constexpr int kMaxN = 32;

template <typename T> struct C2;
template <> struct C2<double> { using type = double2; };
template <> struct C2<float> { using type = float2; };
template <typename T> using c2_t = typename C2<T>::type;

// Geometry of one handle, passed to kernels by value.
struct Geom {
    int N, h, M;          // h = N/2, M = N^3
    int TS, TSp;          // valid (m3,k3) pairs per tile = 3N^2/4; padded to a multiple of 4
    double L, dv, dz;     // half-width, velocity and Fourier spacings
    double lambda;
    int off[kMaxN + 1];   // off[m3]: first pair of row m3 inside a tile (rows ordered by m3)
};

__host__ __device__ inline int kmin_of(int m3, int h) { return m3 - h > 0 ? m3 - h : 0; }
__host__ __device__ inline int kmax_of(int m3, int h, int N) { return m3 + h - 1 < N - 1 ? m3 + h - 1 : N - 1; }

struct Handle {
    int device = 0;
    int precision = CS_FP64;
    Geom g{};
    // weights
    void *ghat = nullptr;         // T[total_tiles * TSp]
    size_t ghat_bytes = 0;
    long long total_tiles = 0;
    int *pencil_tile0 = nullptr;  // device int[N*N + 1]: first tile of each pencil
    // transforms: twiddles exp(-i 2 pi ((k-h)(j-h) mod N) / N), [k][j]
    double2 *tw64 = nullptr;
    float2 *tw32 = nullptr;
    // projection
    double cct_inv[25] = {};
    // workspace
    int ws_cells = 0;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    // pieces of the workspace (set by layout_workspace)
    void *F = nullptr, *Qh = nullptr, *X = nullptr, *Y = nullptr;
    double *Qt = nullptr, *f1 = nullptr, *r1 = nullptr, *scal = nullptr;
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

inline size_t elem_bytes(int precision) { return precision == CS_FP32 ? 4 : 8; }
inline int ngroups_of(int ncells) { return (ncells + kGroup - 1) / kGroup; }

// ---- weights.cu
long long count_tiles(int N, int *pencil_tile0_host /* may be null, size N*N+1 */);
int build_weights(Handle &hd, cudaStream_t s);
int sample_weights(Handle &hd, const int *km_host, int n, double *out_host);

// ---- transform.cu
int launch_forward(const Handle &hd, const double *f, int ncells, cudaStream_t s);   // f -> hd.F
int launch_inverse(const Handle &hd, int ncells, double scale_eps, double *Qt, cudaStream_t s);  // hd.Qh -> Qt
int launch_spectral_to_natural(const Handle &hd, const void *src, int ncells, double *dst, cudaStream_t s);
int launch_natural_to_spectral(const Handle &hd, const double *src, int ncells, void *dst, cudaStream_t s);

// ---- convolve.cu
int launch_convolve(const Handle &hd, int ncells, cudaStream_t s);  // hd.F -> hd.Qh

// ---- conserve.cu
// out = a*x + b*y + c*(P Qt)   (P = projection if project, else identity), per cell
// x, y may be null when a, b are 0.  out may alias Qt, x or y elementwise.
int launch_conserve(const Handle &hd, const double *Qt, int ncells, int project, double a,
                    const double *x, double b, const double *y, double c, double *out,
                    double *moments, cudaStream_t s);
int launch_moments(const Handle &hd, const double *f, int ncells, double *out, cudaStream_t s);

// ---- transport.cu
// out = a*x + b*y + c*rhs(fin)   with rhs the finite-volume transport operator
int launch_transport_stage(const Handle &hd, const double *fin, int ncells, const cs_domain &dom,
                           double a, const double *x, double b, const double *y, double c,
                           double *out, cudaStream_t s);

}  // namespace cs

// The opaque handle of the C ABI.
struct cs_handle_s {
    cs::Handle h;
};
