// K1 / K3: forward and inverse transforms of Sec. 3.2 with the unitary
// normalisation of Sec. 2.2,
//   fhat_k = (2 pi)^{-3/2} dv^3    sum_j f_j    exp(-i zeta_k . v_j),
//   Qt_j   = Re (2 pi)^{-3/2} dzeta^3 sum_k Qhat_k exp(+i zeta_k . v_j) / eps,
// evaluated axis by axis (the 3-D kernel is a product of per-axis factors
// exp(-i 2 pi (k - N/2)(j - N/2) / N)).  Each block transforms one line of
// 32 cells (one cell group) along one axis: the line is staged in shared
// memory and every thread produces one output point of one cell.
//
// Forward:  f (caller layout) --axis 3--> X --axis 2--> Y --axis 1 (x c_f)--> F
// Inverse:  Qh --axis 1--> X --axis 2--> Y --axis 3 (real part x c_i / eps)--> Qt
// so the caller-layout arrays are always read and written along contiguous
// rows.  X, Y, F and Qh use the grouped layout [group][i1][i2][i3][32].
// A block has 32 min(N, 32) threads; for N > 32 each thread produces the
// outputs t, t + 32, ... of its line.
#include "cs_internal.cuh"

namespace cs {

namespace {

__device__ __forceinline__ size_t grouped_index(int N, int g, int i1, int i2, int i3, int lane)
{
    return ((((size_t)g * N + i1) * N + i2) * N + i3) * kGroup + lane;
}

__host__ __device__ inline int line_threads(int N) { return kGroup * (N < 32 ? N : 32); }

// axis-3 transform of the real rows f[c][j1][j2][:]; one block per
// (group, j1, j2).  Cells >= ncells are zero.
template <typename T>
__global__ void forward_rows_kernel(int N, const double *__restrict__ f, int ncells,
                                    const c2_t<T> *__restrict__ tw, c2_t<T> *__restrict__ X)
{
    extern __shared__ unsigned char smem_raw[];
    T *line = reinterpret_cast<T *>(smem_raw);  // [N][32]
    const int bid = blockIdx.x;
    const int j2 = bid % N, j1 = (bid / N) % N, g = bid / (N * N);
    const int tid = threadIdx.x;
    const size_t M = (size_t)N * N * N;
    for (int e = tid; e < kGroup * N; e += blockDim.x) {  // consecutive threads read consecutive j3 of a row
        const int lane = e / N, j3 = e % N;
        const int c = g * kGroup + lane;
        T v = T(0);
        if (c < ncells) v = (T)f[(size_t)c * M + ((size_t)j1 * N + j2) * N + j3];
        line[j3 * kGroup + lane] = v;
    }
    __syncthreads();
    const int lane = tid % kGroup;
    for (int k3 = tid / kGroup; k3 < N; k3 += blockDim.x / kGroup) {
        T re = T(0), im = T(0);
        for (int j = 0; j < N; ++j) {
            const c2_t<T> w = tw[k3 * N + j];
            const T v = line[j * kGroup + lane];
            re += v * w.x;
            im += v * w.y;
        }
        c2_t<T> o;
        o.x = re;
        o.y = im;
        X[grouped_index(N, g, j1, j2, k3, lane)] = o;
    }
}

// axis 1 or 2 of a grouped complex array, one block per line (group, a, b);
// conj != 0 selects exp(+i ...); out = scale * transform(in)
template <typename T>
__global__ void line_kernel(int N, int axis, int conj, T scale, const c2_t<T> *__restrict__ tw,
                            const c2_t<T> *__restrict__ in, c2_t<T> *__restrict__ out)
{
    extern __shared__ unsigned char smem_raw[];
    c2_t<T> *line = reinterpret_cast<c2_t<T> *>(smem_raw);  // [N][32]
    const int bid = blockIdx.x;
    const int b = bid % N, a = (bid / N) % N, g = bid / (N * N);
    const int tid = threadIdx.x;
    const int lane = tid % kGroup, tstep = blockDim.x / kGroup;
    auto index = [&](int t) { return axis == 1 ? grouped_index(N, g, t, a, b, lane) : grouped_index(N, g, a, t, b, lane); };
    for (int t = tid / kGroup; t < N; t += tstep) line[t * kGroup + lane] = in[index(t)];
    __syncthreads();
    const T sgn = conj ? T(-1) : T(1);
    for (int t = tid / kGroup; t < N; t += tstep) {
        T re = T(0), im = T(0);
        for (int j = 0; j < N; ++j) {
            const c2_t<T> w = tw[t * N + j];
            const T wy = sgn * w.y;
            const c2_t<T> v = line[j * kGroup + lane];
            re += v.x * w.x - v.y * wy;
            im += v.x * wy + v.y * w.x;
        }
        c2_t<T> o;
        o.x = scale * re;
        o.y = scale * im;
        out[index(t)] = o;
    }
}

// last inverse pass: axis 3, real part, written to the caller layout rows
template <typename T>
__global__ void inverse_rows_kernel(int N, double scale, const c2_t<T> *__restrict__ tw,
                                    const c2_t<T> *__restrict__ Y, int ncells, double *__restrict__ Qt)
{
    extern __shared__ unsigned char smem_raw[];
    c2_t<T> *line = reinterpret_cast<c2_t<T> *>(smem_raw);  // [N][32]
    double *outl = reinterpret_cast<double *>(line + N * kGroup);  // [32][N]
    const int bid = blockIdx.x;
    const int j2 = bid % N, j1 = (bid / N) % N, g = bid / (N * N);
    const int tid = threadIdx.x;
    const size_t M = (size_t)N * N * N;
    const int lane = tid % kGroup, tstep = blockDim.x / kGroup;
    for (int k3 = tid / kGroup; k3 < N; k3 += tstep) line[k3 * kGroup + lane] = Y[grouped_index(N, g, j1, j2, k3, lane)];
    __syncthreads();
    for (int j3 = tid / kGroup; j3 < N; j3 += tstep) {
        T re = T(0);
        // Re sum_k Y_k exp(+i theta_jk) = sum_k (Y.x cos - Y.y * (+sin)); tw holds exp(-i theta)
        for (int k = 0; k < N; ++k) {
            const c2_t<T> w = tw[k * N + j3];
            const c2_t<T> v = line[k * kGroup + lane];
            re += v.x * w.x + v.y * w.y;
        }
        outl[lane * N + j3] = scale * (double)re;
    }
    __syncthreads();
    for (int e = tid; e < kGroup * N; e += blockDim.x) {  // consecutive threads write consecutive j3 of a row
        const int ln = e / N, j3 = e % N;
        const int c = g * kGroup + ln;
        if (c < ncells) Qt[(size_t)c * M + ((size_t)j1 * N + j2) * N + j3] = outl[ln * N + j3];
    }
}

template <typename T>
__global__ void to_natural_kernel(int N, const c2_t<T> *__restrict__ src, int ncells, double *__restrict__ dst)
{
    const size_t M = (size_t)N * N * N;
    const size_t n = M * ncells;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t c = i / M, k = i % M;
        const size_t j = ((c / kGroup) * M + k) * kGroup + (c % kGroup);
        const c2_t<T> v = src[j];
        dst[2 * i] = (double)v.x;
        dst[2 * i + 1] = (double)v.y;
    }
}

template <typename T>
__global__ void from_natural_kernel(int N, const double *__restrict__ src, int ncells, c2_t<T> *__restrict__ dst)
{
    const size_t M = (size_t)N * N * N;
    const size_t ng = (size_t)(ncells + kGroup - 1) / kGroup;
    const size_t n = ng * M * kGroup;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t lane = i % kGroup, k = (i / kGroup) % M, g = i / (kGroup * M);
        const size_t c = g * kGroup + lane;
        c2_t<T> v;
        v.x = T(0);
        v.y = T(0);
        if (c < (size_t)ncells) {
            v.x = (T)src[2 * (c * M + k)];
            v.y = (T)src[2 * (c * M + k) + 1];
        }
        dst[i] = v;
    }
}

template <typename T>
int forward_impl(const Handle &hd, const double *f, int ncells, cudaStream_t s)
{
    const int N = hd.g.N;
    const int ng = ngroups_of(ncells);
    const unsigned blocks = (unsigned)(ng * N * N);
    const int threads = line_threads(N);
    const c2_t<T> *tw = (const c2_t<T> *)(sizeof(T) == 8 ? (const void *)hd.tw64 : (const void *)hd.tw32);
    const double cf = pow(2.0 * M_PI, -1.5) * hd.g.dv * hd.g.dv * hd.g.dv;
    forward_rows_kernel<T><<<blocks, threads, sizeof(T) * N * kGroup, s>>>(N, f, ncells, tw, (c2_t<T> *)hd.X);
    line_kernel<T><<<blocks, threads, sizeof(c2_t<T>) * N * kGroup, s>>>(N, 2, 0, T(1), tw, (const c2_t<T> *)hd.X,
                                                                          (c2_t<T> *)hd.Y);
    line_kernel<T><<<blocks, threads, sizeof(c2_t<T>) * N * kGroup, s>>>(N, 1, 0, (T)cf, tw, (const c2_t<T> *)hd.Y,
                                                                          (c2_t<T> *)hd.F);
    CS_LAUNCHED(3, s, "forward transform");
    return CS_OK;
}

template <typename T>
int inverse_impl(const Handle &hd, int ncells, double eps, double *Qt, cudaStream_t s)
{
    const int N = hd.g.N;
    const int ng = ngroups_of(ncells);
    const unsigned blocks = (unsigned)(ng * N * N);
    const int threads = line_threads(N);
    const c2_t<T> *tw = (const c2_t<T> *)(sizeof(T) == 8 ? (const void *)hd.tw64 : (const void *)hd.tw32);
    const double ci = pow(2.0 * M_PI, -1.5) * hd.g.dz * hd.g.dz * hd.g.dz / eps;
    line_kernel<T><<<blocks, threads, sizeof(c2_t<T>) * N * kGroup, s>>>(N, 1, 1, T(1), tw, (const c2_t<T> *)hd.Qh,
                                                                          (c2_t<T> *)hd.X);
    line_kernel<T><<<blocks, threads, sizeof(c2_t<T>) * N * kGroup, s>>>(N, 2, 1, T(1), tw, (const c2_t<T> *)hd.X,
                                                                          (c2_t<T> *)hd.Y);
    const size_t sm = sizeof(c2_t<T>) * N * kGroup + sizeof(double) * N * kGroup;
    inverse_rows_kernel<T><<<blocks, threads, sm, s>>>(N, ci, tw, (const c2_t<T> *)hd.Y, ncells, Qt);
    CS_LAUNCHED(3, s, "inverse transform");
    return CS_OK;
}

}  // namespace

int launch_forward(const Handle &hd, const double *f, int ncells, cudaStream_t s)
{
    if (fused_available(hd)) return launch_forward_fused(hd, f, ncells, s);
    return hd.precision == CS_FP32 ? forward_impl<float>(hd, f, ncells, s) : forward_impl<double>(hd, f, ncells, s);
}

int launch_inverse(const Handle &hd, int ncells, double eps, double *Qt, cudaStream_t s)
{
    if (fused_available(hd))
        return launch_inverse_project(hd, ncells, eps, 0, 0.0, nullptr, 0.0, nullptr, 1.0, Qt, s);
    return hd.precision == CS_FP32 ? inverse_impl<float>(hd, ncells, eps, Qt, s)
                                   : inverse_impl<double>(hd, ncells, eps, Qt, s);
}

int launch_spectral_to_natural(const Handle &hd, const void *src, int ncells, double *dst, cudaStream_t s)
{
    const int N = hd.g.N;
    if (hd.precision == CS_FP32)
        to_natural_kernel<float><<<1024, 256, 0, s>>>(N, (const float2 *)src, ncells, dst);
    else
        to_natural_kernel<double><<<1024, 256, 0, s>>>(N, (const double2 *)src, ncells, dst);
    CS_LAUNCHED(1, s, "spectral layout conversion");
    return CS_OK;
}

int launch_natural_to_spectral(const Handle &hd, const double *src, int ncells, void *dst, cudaStream_t s)
{
    const int N = hd.g.N;
    if (hd.precision == CS_FP32)
        from_natural_kernel<float><<<1024, 256, 0, s>>>(N, src, ncells, (float2 *)dst);
    else
        from_natural_kernel<double><<<1024, 256, 0, s>>>(N, src, ncells, (double2 *)dst);
    CS_LAUNCHED(1, s, "spectral layout conversion");
    return CS_OK;
}

}  // namespace cs
