// K4: the conservation step of Sec. 3.3 in double precision.  With the
// integration matrix C (rows dv^3 (1, v1, v2, v3, |v|^2)) the constrained
// least-squares solution is Q = Qt - C^T (C C^T)^{-1} C Qt; (C C^T)^{-1} is a
// 5x5 constant of the handle.  One block per cell: the five moments are
// reduced with warp shuffles, the 5x5 product is done by one thread, and the
// correction is applied together with the Runge-Kutta combination of the
// caller (out = a x + b y + c Q), so a Heun stage costs no extra pass.
#include <algorithm>

#include "cs_internal.cuh"

namespace cs {

namespace {

constexpr int kThreads = 256;

struct Proj {
    double ainv[25];
};

__device__ __forceinline__ void c_row(const Geom &g, int j, double r[5])
{
    const int N = g.N, h = g.h;
    const double w = g.dv * g.dv * g.dv;
    const double v1 = g.dv * (j / (N * N) - h);
    const double v2 = g.dv * ((j / N) % N - h);
    const double v3 = g.dv * (j % N - h);
    r[0] = w;
    r[1] = w * v1;
    r[2] = w * v2;
    r[3] = w * v3;
    r[4] = w * (v1 * v1 + v2 * v2 + v3 * v3);
}

// block-wide sum of 5 doubles; result valid in every thread
__device__ void block_sum5(double v[5], double *sh /* [5][kThreads/32] */)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        double x = v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[i * 32 + wid] = x;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        double x = 0;
        for (int k = 0; k < nw; ++k) x += sh[i * 32 + k];
        v[i] = x;
    }
    __syncthreads();
}

// v_k = dv (k - N/2) and its square, per axis, in shared memory: the double
// work per point is then 7 operations for the moments and 9 for the update
__device__ __forceinline__ void fill_axis(const Geom &g, double *va, double *v2a)
{
    for (int i = threadIdx.x; i < g.N; i += blockDim.x) {
        const double v = g.dv * (i - g.h);
        va[i] = v;
        v2a[i] = v * v;
    }
}

// Double precision runs at 1/64 of float here, so a cell is spread over
// `parts` blocks: moments_part_kernel writes one partial 5-vector per block,
// apply_kernel sums a cell's partials in a fixed order (deterministic),
// forms y = (C C^T)^{-1} C Qt and writes out = a x + b y + c (Qt - C^T y).
__global__ void __launch_bounds__(kThreads) moments_part_kernel(Geom g, const double *__restrict__ Qt, int parts,
                                                                double *__restrict__ partial)
{
    __shared__ double sh[5 * 32];
    __shared__ double va[kMaxN], v2a[kMaxN];
    fill_axis(g, va, v2a);
    __syncthreads();
    const int N = g.N, NN = g.N * g.N;
    const int cell = blockIdx.x / parts, part = blockIdx.x % parts;
    const int chunk = (g.M + parts - 1) / parts;
    const int j0 = part * chunk, j1 = min(g.M, j0 + chunk);
    const size_t base = (size_t)cell * g.M;
    double mom[5] = {0, 0, 0, 0, 0};
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const int i1 = j / NN, i2 = (j / N) % N, i3 = j % N;
        const double q = Qt[base + j];
        mom[0] += q;
        mom[1] = fma(va[i1], q, mom[1]);
        mom[2] = fma(va[i2], q, mom[2]);
        mom[3] = fma(va[i3], q, mom[3]);
        mom[4] = fma(v2a[i1] + v2a[i2] + v2a[i3], q, mom[4]);
    }
    block_sum5(mom, sh);
    if (threadIdx.x < 5) partial[(size_t)blockIdx.x * 5 + threadIdx.x] = mom[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads) apply_kernel(Geom g, Proj pj, const double *Qt, int project, int parts,
                                                         const double *__restrict__ partial, double a,
                                                         const double *x, double b, const double *y, double c,
                                                         double *out, double *moments)
{
    __shared__ double va[kMaxN], v2a[kMaxN];
    __shared__ double ycoef[5];
    fill_axis(g, va, v2a);
    const int N = g.N, NN = g.N * g.N;
    const int cell = blockIdx.x / parts, part = blockIdx.x % parts;
    const double w = g.dv * g.dv * g.dv;
    if (threadIdx.x == 0) {
        double mom[5] = {0, 0, 0, 0, 0};
        if (project || moments)
            for (int q = 0; q < parts; ++q)
                for (int i = 0; i < 5; ++i) mom[i] += partial[((size_t)cell * parts + q) * 5 + i];
        for (int i = 0; i < 5; ++i) {
            mom[i] *= w;
            if (moments && part == 0) moments[5 * (size_t)cell + i] = mom[i];
        }
        for (int i = 0; i < 5; ++i) {
            double s = 0;
            if (project)
                for (int k = 0; k < 5; ++k) s += pj.ainv[5 * i + k] * mom[k];
            ycoef[i] = w * s;  // C^T y = w (1, v1, v2, v3, |v|^2) . y
        }
    }
    __syncthreads();
    const double y0 = ycoef[0], y1 = ycoef[1], y2 = ycoef[2], y3 = ycoef[3], y4 = ycoef[4];
    const int chunk = (g.M + parts - 1) / parts;
    const int j0 = part * chunk, j1 = min(g.M, j0 + chunk);
    const size_t base = (size_t)cell * g.M;
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const int i1 = j / NN, i2 = (j / N) % N, i3 = j % N;
        double q = Qt[base + j];
        if (project) {
            const double corr = fma(y4, v2a[i1] + v2a[i2] + v2a[i3],
                                    fma(y3, va[i3], fma(y2, va[i2], fma(y1, va[i1], y0))));
            q -= corr;
        }
        double o = c * q;
        if (x) o = fma(a, x[base + j], o);
        if (y) o = fma(b, y[base + j], o);
        out[base + j] = o;
    }
}

__global__ void __launch_bounds__(kThreads) moments_kernel(Geom g, const double *__restrict__ f,
                                                           double *__restrict__ out)
{
    __shared__ double sh[5 * 32];
    const int cell = blockIdx.x;
    const size_t base = (size_t)cell * g.M;
    double mom[5] = {0, 0, 0, 0, 0};
    for (int j = threadIdx.x; j < g.M; j += blockDim.x) {
        double r[5];
        c_row(g, j, r);
        const double v = f[base + j];
#pragma unroll
        for (int i = 0; i < 5; ++i) mom[i] += r[i] * v;
    }
    block_sum5(mom, sh);
    if (threadIdx.x == 0)
        for (int i = 0; i < 5; ++i) out[5 * (size_t)cell + i] = mom[i];
}

// The input scan of CS_TUNE_CHECK_INPUT (failure detection, no counterpart
// in the paper): one pass over the distribution; a warp that meets a
// non-finite value sets bit 1 of the handle's status word, with `negative`
// a negative value bit 2.  Grid-stride loop, one atomic per warp at most.
__global__ void __launch_bounds__(kThreads) input_check_kernel(const double *__restrict__ f, long long count,
                                                               int negative, int *err)
{
    int bits = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const double v = f[i];
        if (!isfinite(v)) bits |= 2;
        else if (negative && v < 0.0) bits |= 4;
    }
    bits = __reduce_or_sync(0xffffffffu, bits);
    if (bits && (threadIdx.x & 31) == 0) atomicOr(err, bits);
}

}  // namespace

int launch_input_check(const Handle &hd, const double *f, long long count, cudaStream_t s)
{
    if (hd.check_input == 0 || count <= 0) return CS_OK;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, hd.device);
    const long long want = (count + kThreads - 1) / kThreads;
    const int blocks = (int)std::min<long long>(want, 4LL * std::max(1, sms));
    input_check_kernel<<<blocks, kThreads, 0, s>>>(f, count, hd.check_input == 2, hd.err);
    CS_LAUNCHED(1, s, "input scan");
    return CS_OK;
}

int conserve_parts(int M) { return M >= 32768 ? 8 : M >= 4096 ? 4 : 1; }

int launch_conserve(const Handle &hd, const double *Qt, int ncells, int project, double a, const double *x,
                    double b, const double *y, double c, double *out, double *moments, cudaStream_t s)
{
    Proj pj;
    for (int i = 0; i < 25; ++i) pj.ainv[i] = hd.cct_inv[i];
    const int parts = conserve_parts(hd.g.M);
    const unsigned blocks = (unsigned)(ncells * parts);
    if (project || moments) moments_part_kernel<<<blocks, kThreads, 0, s>>>(hd.g, Qt, parts, hd.part5);
    apply_kernel<<<blocks, kThreads, 0, s>>>(hd.g, pj, Qt, project, parts, hd.part5, a, x, b, y, c, out, moments);
    CS_LAUNCHED((project || moments) ? 2 : 1, s, "conservation projection");
    return CS_OK;
}

int launch_moments(const Handle &hd, const double *f, int ncells, double *out, cudaStream_t s)
{
    moments_kernel<<<ncells, kThreads, 0, s>>>(hd.g, f, out);
    CS_LAUNCHED(1, s, "moments");
    return CS_OK;
}

}  // namespace cs
