// Whole-cell transforms for float handles with N <= 16, where one cell's
// spectrum (N^3 complex floats, 32 KB at N = 16) fits in shared memory.
//
// forward_fused_kernel: one block per cell.  The cell's f is read once
// (contiguous), the three axis passes of the forward transform of Sec. 3.2,
//   fhat_k = (2 pi)^{-3/2} dv^3 sum_j f_j exp(-i zeta_k . v_j),
// run in shared memory (one line of N points per thread, twiddles broadcast
// from shared memory), and fhat goes out in the 32-cell grouped layout the
// convolution reads.
//
// inverse_project_kernel: one block per cell.  Reads Qhat of the cell, runs
// the three inverse passes (Qt = Re (2 pi)^{-3/2} dzeta^3 sum_k ... / eps),
// then the conservation projection of Sec. 3.3 in double precision and the
// caller's Runge-Kutta combination, out = a x + b y + c (Qt - C^T y), with
// y = (C C^T)^{-1} C Qt.  The moments and the correction are factorised per
// line (fixed v1, v2): per point 3 double operations for C Qt and 5 for the
// update, since double precision is the scarce unit on this part.
//
// Shared-memory layout of a cell: element (i1, i2, i3) at (i1 N + i2)(N + 1) + i3;
// the +1 pad keeps the three line directions free of bank conflicts.
#include "cs_internal.cuh"

namespace cs {

namespace {

constexpr int kFusedThreads = 256;

struct Proj5 {
    double ainv[25];
};

__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// one line of N points at X[base + stride * i], transformed in place with the
// twiddles T (exp(-i...) ; conj selects exp(+i...)), scaled by `scale`
template <int N>
__device__ __forceinline__ void line_dft(float2 *X, int base, int stride, const float2 *T, bool conj, float scale)
{
    float2 v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = X[base + stride * j];
#pragma unroll 1
    for (int k = 0; k < N; ++k) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            float2 w = T[k * N + j];
            if (conj) w.y = -w.y;
            const float2 p = cmulf(v[j], w);
            acc.x += p.x;
            acc.y += p.y;
        }
        X[base + stride * k] = make_float2(scale * acc.x, scale * acc.y);
    }
}

template <int N>
__global__ void __launch_bounds__(kFusedThreads) forward_fused_kernel(const double *__restrict__ f, int ncells,
                                                                      const float2 *__restrict__ tw, float cf,
                                                                      float2 *__restrict__ F)
{
    constexpr int M = N * N * N, P = N + 1, LINES = N * N;
    extern __shared__ float2 X[];      // [N*N][P]
    __shared__ float2 T[N * N];
    const int cell = blockIdx.x;
    const int tid = threadIdx.x;
    for (int i = tid; i < N * N; i += blockDim.x) T[i] = tw[i];
    const bool real = cell < ncells;
    for (int j = tid; j < M; j += blockDim.x)
        X[(j / N) * P + j % N] = make_float2(real ? (float)f[(size_t)cell * M + j] : 0.f, 0.f);
    __syncthreads();
    for (int l = tid; l < LINES; l += blockDim.x) line_dft<N>(X, l * P, 1, T, false, 1.f);           // axis 3
    __syncthreads();
    for (int l = tid; l < LINES; l += blockDim.x) line_dft<N>(X, (l / N) * N * P + l % N, P, T, false, 1.f);  // axis 2
    __syncthreads();
    for (int l = tid; l < LINES; l += blockDim.x) line_dft<N>(X, (l / N) * P + l % N, N * P, T, false, cf);   // axis 1
    __syncthreads();
    const int g = cell / kGroup, lane = cell % kGroup;
    for (int k = tid; k < M; k += blockDim.x)
        F[((size_t)g * M + k) * kGroup + lane] = X[(k / N) * P + k % N];
}

template <int N>
__global__ void __launch_bounds__(kFusedThreads) inverse_project_kernel(
    const float2 *__restrict__ Qh, const float2 *__restrict__ tw, float ci, double dv, int project, Proj5 pj,
    double a, const double *x, double b, const double *y, double c, double *out, double *moments)
{
    constexpr int M = N * N * N, P = N + 1, LINES = N * N, H = N / 2;
    extern __shared__ float2 X[];      // [N*N][P]; after the transform, reused as double Qt
    __shared__ float2 T[N * N];
    __shared__ double vax[N], lbase[N * N];
    __shared__ double red[5][kFusedThreads / 32];
    __shared__ double ycoef[5];
    const int cell = blockIdx.x;
    const int g = cell / kGroup, lane = cell % kGroup;
    const int tid = threadIdx.x;
    for (int i = tid; i < N * N; i += blockDim.x) T[i] = tw[i];
    if (tid < N) vax[tid] = dv * (tid - H);
    for (int k = tid; k < M; k += blockDim.x) X[(k / N) * P + k % N] = Qh[((size_t)g * M + k) * kGroup + lane];
    __syncthreads();
    for (int l = tid; l < LINES; l += blockDim.x) line_dft<N>(X, (l / N) * P + l % N, N * P, T, true, 1.f);   // axis 1
    __syncthreads();
    for (int l = tid; l < LINES; l += blockDim.x) line_dft<N>(X, (l / N) * N * P + l % N, P, T, true, 1.f);  // axis 2
    __syncthreads();
    // axis 3, keeping the real part as a double in the same slot
    double *Qd = reinterpret_cast<double *>(X);
    for (int l = tid; l < LINES; l += blockDim.x) {
        float2 v[N];
#pragma unroll
        for (int j = 0; j < N; ++j) v[j] = X[l * P + j];
#pragma unroll 1
        for (int k = 0; k < N; ++k) {
            float re = 0.f;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const float2 w = T[j * N + k];  // exp(-i theta); Re(v exp(+i theta)) = v.x w.x + v.y w.y
                re = fmaf(v[j].x, w.x, fmaf(v[j].y, w.y, re));
            }
            Qd[l * P + k] = (double)(ci * re);
        }
    }
    __syncthreads();
    // moments, per line (j1, j2): S0 = sum q, S3 = sum v3 q, S33 = sum v3^2 q
    double m[5] = {0, 0, 0, 0, 0};
    if (project || moments) {
        for (int l = tid; l < LINES; l += blockDim.x) {
            double s0 = 0, s3 = 0, s33 = 0;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const double q = Qd[l * P + j], v3 = vax[j];
                s0 += q;
                s3 = fma(v3, q, s3);
                s33 = fma(v3 * v3, q, s33);
            }
            const double v1 = vax[l / N], v2 = vax[l % N];
            m[0] += s0;
            m[1] = fma(v1, s0, m[1]);
            m[2] = fma(v2, s0, m[2]);
            m[3] += s3;
            m[4] += fma(v1 * v1 + v2 * v2, s0, s33);
        }
        const int w = tid >> 5, ln = tid & 31;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            double t = m[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (ln == 0) red[i][w] = t;
        }
    }
    __syncthreads();
    if (tid == 0) {
        const double w3 = dv * dv * dv;
        double mom[5];
        for (int i = 0; i < 5; ++i) {
            double t = 0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[i][k];
            mom[i] = (project || moments) ? w3 * t : 0.0;
            if (moments) moments[5 * (size_t)cell + i] = mom[i];
        }
        for (int i = 0; i < 5; ++i) {
            double s = 0;
            if (project)
                for (int k = 0; k < 5; ++k) s += pj.ainv[5 * i + k] * mom[k];
            ycoef[i] = w3 * s;  // C^T y = w3 (1, v1, v2, v3, |v|^2) . y
        }
    }
    __syncthreads();
    const double y0 = ycoef[0], y1 = ycoef[1], y2 = ycoef[2], y3 = ycoef[3], y4 = ycoef[4];
    for (int l = tid; l < LINES; l += blockDim.x) {
        const double v1 = vax[l / N], v2 = vax[l % N];
        lbase[l] = fma(y4, v1 * v1 + v2 * v2, fma(y2, v2, fma(y1, v1, y0)));
    }
    __syncthreads();
    const size_t base = (size_t)cell * M;
    for (int j = tid; j < M; j += blockDim.x) {
        const int l = j / N, j3 = j % N;
        const double v3 = vax[j3];
        double q = Qd[l * P + j3];
        if (project) q -= lbase[l] + v3 * fma(y4, v3, y3);
        double o = c * q;
        if (x) o = fma(a, x[base + j], o);
        if (y) o = fma(b, y[base + j], o);
        out[base + j] = o;
    }
}

template <int N>
size_t fused_smem() { return sizeof(float2) * (size_t)N * N * (N + 1); }

template <int N>
int forward_n(const Handle &hd, const double *f, int ncells, cudaStream_t s)
{
    const float cf = (float)(pow(2.0 * M_PI, -1.5) * hd.g.dv * hd.g.dv * hd.g.dv);
    const unsigned blocks = (unsigned)(ngroups_of(ncells) * kGroup);
    forward_fused_kernel<N><<<blocks, kFusedThreads, fused_smem<N>(), s>>>(f, ncells, hd.tw32, cf, (float2 *)hd.F);
    CS_LAUNCHED(1, s, "forward transform (fused)");
    return CS_OK;
}

template <int N>
int inverse_n(const Handle &hd, int ncells, double eps, int project, double a, const double *x, double b,
              const double *y, double c, double *out, double *moments, cudaStream_t s)
{
    Proj5 pj;
    for (int i = 0; i < 25; ++i) pj.ainv[i] = hd.cct_inv[i];
    const float ci = (float)(pow(2.0 * M_PI, -1.5) * hd.g.dz * hd.g.dz * hd.g.dz / eps);
    inverse_project_kernel<N><<<ncells, kFusedThreads, fused_smem<N>(), s>>>(
        (const float2 *)hd.Qh, hd.tw32, ci, hd.g.dv, project, pj, a, x, b, y, c, out, moments);
    CS_LAUNCHED(1, s, "inverse transform and projection (fused)");
    return CS_OK;
}

}  // namespace

bool fused_available(const Handle &hd)
{
    return hd.precision == CS_FP32 && (hd.g.N == 8 || hd.g.N == 12 || hd.g.N == 16);
}

int launch_forward_fused(const Handle &hd, const double *f, int ncells, cudaStream_t s)
{
    switch (hd.g.N) {
    case 8: return forward_n<8>(hd, f, ncells, s);
    case 12: return forward_n<12>(hd, f, ncells, s);
    case 16: return forward_n<16>(hd, f, ncells, s);
    default: return set_error(CS_ENOTSUP, "fused forward transform: unsupported N");
    }
}

int launch_inverse_project(const Handle &hd, int ncells, double eps, int project, double a, const double *x,
                           double b, const double *y, double c, double *out, double *moments, cudaStream_t s)
{
    switch (hd.g.N) {
    case 8: return inverse_n<8>(hd, ncells, eps, project, a, x, b, y, c, out, moments, s);
    case 12: return inverse_n<12>(hd, ncells, eps, project, a, x, b, y, c, out, moments, s);
    case 16: return inverse_n<16>(hd, ncells, eps, project, a, x, b, y, c, out, moments, s);
    default: return set_error(CS_ENOTSUP, "fused inverse transform: unsupported N");
    }
}

}  // namespace cs
