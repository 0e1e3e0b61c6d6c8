// Whole-cell transforms for float handles with N <= 24, where one cell's
// spectrum (N^3 complex floats, 32 KB at N = 16, 113 KB at N = 24) fits in
// shared memory.
//
// forward_fused_kernel: one block per cell.  The cell's f is read once
// (contiguous), the three axis passes of the forward transform of Sec. 3.2,
//   fhat_k = (2 pi)^{-3/2} dv^3 sum_j f_j exp(-i zeta_k . v_j),
// run in shared memory, and fhat goes out in the 32-cell grouped layout the
// convolution reads.
//
// inverse_project_kernel: one block per cell.  Reads Qhat of the cell (the
// sum of the convolution's partial sums, when it leaves two), runs the three
// inverse passes (Qt = Re (2 pi)^{-3/2} dzeta^3 sum_k ... / eps), then the
// conservation projection of Sec. 3.3 in double precision and the caller's
// Runge-Kutta combination,
//   out = a x + b y + P(c Qt),  P(q) = q - C^T (C C^T)^{-1} C q.
// The step factor c is folded into the float scale of the last inverse pass,
// so the projection works on c Qt directly (P is linear; the moments and the
// correction use the same doubles, so the projected values conserve exactly
// up to rounding).  The moments and the correction are factorised per line
// (fixed v1, v2): per point 3 double operations for C q and 4 for the update,
// since double precision is the scarce unit on this part.
//
// Line transforms.  Along one axis, with h = N/2 and the grid indices of
// Sec. 3.1, exp(-2 pi i (k-h)(j-h)/N) = (-1)^{k+j} (-1)^h exp(-2 pi i k j/N)
// and (-1)^h = 1 for the even h used here, so the shifted transform is a plain
// length-N DFT with the odd inputs and the odd outputs negated (sign flips
// only).  The DFT runs in registers as a two-level Cooley-Tukey FFT,
// N = 4 x (N/4): length-4 and length-N/4 DFTs (2, 3 or 4 points) with
// twiddles that are compile-time constants (cos and sin of multiples of a
// 48th of a turn, which covers N = 8, 12, 16, 24).  One thread owns one line, so
// the passes need no synchronisation inside a pass.
//
// Shared-memory layout of a cell: element (i1, i2, i3) at (i1 N + i2)(N + 1) + i3;
// the +1 pad keeps the three line directions free of bank conflicts.
#include <algorithm>

#include "cs_internal.cuh"

namespace cs {

namespace {

// cos(2 pi e / 48) for e = 0 .. 12 (a quarter turn); other angles by symmetry
__host__ __device__ constexpr float cos48q(int e)
{
    return e == 0    ? 1.0f
           : e == 1  ? 0.991444861f
           : e == 2  ? 0.965925826f
           : e == 3  ? 0.923879533f
           : e == 4  ? 0.866025404f
           : e == 5  ? 0.793353340f
           : e == 6  ? 0.707106781f
           : e == 7  ? 0.608761429f
           : e == 8  ? 0.5f
           : e == 9  ? 0.382683432f
           : e == 10 ? 0.258819045f
           : e == 11 ? 0.130526192f
                     : 0.0f;
}

__host__ __device__ constexpr float cos48(int e)
{
    return e <= 12 ? cos48q(e) : e <= 24 ? -cos48q(24 - e) : e <= 36 ? -cos48q(e - 24) : cos48q(48 - e);
}

__host__ __device__ constexpr float sin48(int e) { return cos48((e + 36) % 48); }  // sin t = cos(t - quarter turn)

// x * w^m with w = exp(-2 pi i / R) (forward) or exp(+2 pi i / R) (inverse),
// m a compile-time value after unrolling; quarter turns are exact swaps
template <int R, bool INV>
__device__ __forceinline__ float2 rot(float2 x, int m)
{
    const int e = (m % R) * (48 / R);
    if (e == 0) return x;
    if (e == 24) return make_float2(-x.x, -x.y);
    if (e == 12) return INV ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
    if (e == 36) return INV ? make_float2(x.y, -x.x) : make_float2(-x.y, x.x);
    const float c = cos48(e), s = INV ? sin48(e) : -sin48(e);
    return make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c));
}

// in place: x[k] <- sum_n x[n] w^{n k}, w = exp(-+2 pi i / N), N = 4 R2
template <int N, bool INV>
__device__ __forceinline__ void fft(float2 (&x)[N])
{
    constexpr int R1 = 4, R2 = N / R1;
    float2 y[N];  // y[n2 R1 + k1]: length-4 DFTs over n1 of x[R2 n1 + n2], twiddled
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            float2 acc = x[n2];
#pragma unroll
            for (int n1 = 1; n1 < R1; ++n1) {
                const float2 t = rot<R1, INV>(x[R2 * n1 + n2], n1 * k1);
                acc.x += t.x;
                acc.y += t.y;
            }
            y[n2 * R1 + k1] = rot<N, INV>(acc, n2 * k1);
        }
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
            float2 acc = y[k1];
#pragma unroll
            for (int n2 = 1; n2 < R2; ++n2) {
                const float2 t = rot<R2, INV>(y[n2 * R1 + k1], n2 * k2);
                acc.x += t.x;
                acc.y += t.y;
            }
            x[k1 + R1 * k2] = acc;
        }
    }
}

// the shifted transform of one line at X[base + stride * j], j = 0..N-1, in
// place, times `scale`: sum_j x_j exp(-+2 pi i (k-h)(j-h)/N)
template <int N, bool INV>
__device__ __forceinline__ void line_transform(float2 *X, int base, int stride, float scale)
{
    float2 v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const float2 t = X[base + stride * j];
        v[j] = (j & 1) ? make_float2(-t.x, -t.y) : t;
    }
    fft<N, INV>(v);
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const float sk = (k & 1) ? -scale : scale;
        X[base + stride * k] = make_float2(sk * v[k].x, sk * v[k].y);
    }
}

// one thread per line, rounded up to whole warps (the reductions shuffle over
// full warps): 64, 160, 256, 576 for N = 8, 12, 16, 24
template <int N>
constexpr int kThreads = (N * N + 31) / 32 * 32 < 64 ? 64 : (N * N + 31) / 32 * 32;

// loops over a cell's N^3 points run kPer<N> rounds of the block, in chunks
// of kChunk<N> rounds unrolled with every global load of a chunk issued
// before its first use (one chunk up to N = 16; at N = 24 three chunks of 8,
// which keeps the registers of a 576-thread block within its share)
template <int N>
constexpr int kPer = (N * N * N + kThreads<N> - 1) / kThreads<N>;
template <int N>
constexpr int kChunk = kPer<N> <= 16 ? kPer<N> : 8;

struct Proj5 {
    double ainv[25];
};

template <int N>
__global__ void __launch_bounds__(kThreads<N>) forward_fused_kernel(const double *__restrict__ f, int ncells, float cf,
                                                                    float2 *__restrict__ F)
{
    constexpr int M = N * N * N, P = N + 1, NT = kThreads<N>, LINES = N * N;
    extern __shared__ float2 X[];  // [N*N][P]
    const int cell = blockIdx.x;
    const int tid = threadIdx.x;
    const bool real = cell < ncells;
    static_assert(kPer<N> % kChunk<N> == 0, "whole chunks");
    for (int r0 = 0; r0 < kPer<N>; r0 += kChunk<N>) {
        double fr[kChunk<N>];
#pragma unroll
        for (int r = 0; r < kChunk<N>; ++r) {
            const int j = (r0 + r) * NT + tid;
            fr[r] = (real && j < M) ? f[(size_t)cell * M + j] : 0.0;
        }
#pragma unroll
        for (int r = 0; r < kChunk<N>; ++r) {
            const int j = (r0 + r) * NT + tid;
            if (j < M) X[(j / N) * P + j % N] = make_float2((float)fr[r], 0.f);
        }
    }
    __syncthreads();
    const int l = tid;
    if (l < LINES) line_transform<N, false>(X, l * P, 1, 1.f);  // axis 3
    __syncthreads();
    if (l < LINES) line_transform<N, false>(X, (l / N) * N * P + l % N, P, 1.f);  // axis 2
    __syncthreads();
    if (l < LINES) line_transform<N, false>(X, (l / N) * P + l % N, N * P, cf);  // axis 1
    __syncthreads();
    const int g = cell / kGroup, lane = cell % kGroup;
#pragma unroll
    for (int r = 0; r < kPer<N>; ++r) {
        const int k = r * NT + tid;
        if (k < M) F[((size_t)g * M + k) * kGroup + lane] = X[(k / N) * P + k % N];
    }
}

template <int N>
__global__ void __launch_bounds__(kThreads<N>) inverse_project_kernel(
    const float2 *__restrict__ Qh, const float2 *__restrict__ Qh2, float cic, double dv, int project, Proj5 pj,
    double a, const double *x, double b, const double *y, double *out)
{
    constexpr int M = N * N * N, P = N + 1, LINES = N * N, H = N / 2, NT = kThreads<N>, NW = NT / 32;
    static_assert(NT % 32 == 0, "whole warps");
    extern __shared__ float2 X[];  // [N*N][P]; after the transform, reused as double q = c Qt
    __shared__ double vax[N], vsq[N], cv3[N], lbase[N * N];
    __shared__ double red[5][NW];
    __shared__ double ycoef[5], mom_s[5];
    const int cell = blockIdx.x;
    const int g = cell / kGroup, lane = cell % kGroup;
    const int tid = threadIdx.x;
    if (tid < N) {
        vax[tid] = dv * (tid - H);
        vsq[tid] = vax[tid] * vax[tid];
    }
    for (int r0 = 0; r0 < kPer<N>; r0 += kChunk<N>) {
        float2 qa[kChunk<N>], qb[kChunk<N>];
#pragma unroll
        for (int r = 0; r < kChunk<N>; ++r) {
            const int k = (r0 + r) * NT + tid;
            const size_t i = ((size_t)g * M + (k < M ? k : 0)) * kGroup + lane;
            qa[r] = Qh[i];
            qb[r] = Qh2 ? Qh2[i] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < kChunk<N>; ++r) {  // two partial sums of the convolution, added in a fixed order
            const int k = (r0 + r) * NT + tid;
            if (k < M) X[(k / N) * P + k % N] = Qh2 ? make_float2(qa[r].x + qb[r].x, qa[r].y + qb[r].y) : qa[r];
        }
    }
    __syncthreads();
    const int l = tid;
    if (l < LINES) line_transform<N, true>(X, (l / N) * P + l % N, N * P, 1.f);  // axis 1
    __syncthreads();
    if (l < LINES) line_transform<N, true>(X, (l / N) * N * P + l % N, P, 1.f);  // axis 2
    __syncthreads();
    // axis 3: c times the real part, as a double in the same slot (one thread
    // owns the line, so reading it whole before writing makes this safe)
    double *Qd = reinterpret_cast<double *>(X);
    double m[5] = {0, 0, 0, 0, 0};
    if (l < LINES) {
        float2 v[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const float2 t = X[l * P + j];
            v[j] = (j & 1) ? make_float2(-t.x, -t.y) : t;
        }
        fft<N, true>(v);
        // moments of the line (j1, j2) = l: S0 = sum q, S3 = sum v3 q, S33 = sum v3^2 q
        double s0 = 0, s3 = 0, s33 = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const double qq = (double)(((k & 1) ? -cic : cic) * v[k].x);
            Qd[l * P + k] = qq;
            s0 += qq;
            s3 = fma(vax[k], qq, s3);
            s33 = fma(vsq[k], qq, s33);
        }
        m[0] = s0;
        m[1] = vax[l / N] * s0;
        m[2] = vax[l % N] * s0;
        m[3] = s3;
        m[4] = fma(vsq[l / N] + vsq[l % N], s0, s33);
    }
    if (project) {
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
    // moments (thread i sums moment i over the warps), then y = (C C^T)^{-1} C q
    // (thread i takes row i); the same order of operations as one thread would use
    const double w3 = dv * dv * dv;
    if (tid < 5) {
        double t = 0;
        if (project)
            for (int k = 0; k < NW; ++k) t += red[tid][k];
        mom_s[tid] = w3 * t;
    }
    __syncthreads();
    if (tid < 5) {
        double s = 0;
        if (project)
            for (int k = 0; k < 5; ++k) s += pj.ainv[5 * tid + k] * mom_s[k];
        ycoef[tid] = w3 * s;  // C^T y = w3 (1, v1, v2, v3, |v|^2) . y
    }
    __syncthreads();
    const double y0 = ycoef[0], y1 = ycoef[1], y2 = ycoef[2], y3 = ycoef[3], y4 = ycoef[4];
    // correction C^T y at (v1, v2, v3) = lbase(v1, v2) + cv3(v3)
    for (int i = tid; i < LINES; i += NT) {
        const double v1 = vax[i / N], v2 = vax[i % N];
        lbase[i] = fma(y4, vsq[i / N] + vsq[i % N], fma(y2, v2, fma(y1, v1, y0)));
    }
    if (tid < N) cv3[tid] = vax[tid] * fma(y4, vax[tid], y3);
    __syncthreads();
    const size_t base = (size_t)cell * M;
    // x and y may alias out (same index, same thread only): a chunk's loads
    // come before its stores
    for (int r0 = 0; r0 < kPer<N>; r0 += kChunk<N>) {
        double xr[kChunk<N>], yr[kChunk<N>];
#pragma unroll
        for (int r = 0; r < kChunk<N>; ++r) {
            const int j = (r0 + r) * NT + tid;
            xr[r] = (x && j < M) ? x[base + j] : 0.0;
            yr[r] = (y && j < M) ? y[base + j] : 0.0;
        }
#pragma unroll
        for (int r = 0; r < kChunk<N>; ++r) {
            const int j = (r0 + r) * NT + tid;
            if (j >= M) break;
            const int jl = j / N, j3 = j % N;
            double o = Qd[jl * P + j3];
            if (project) o -= lbase[jl] + cv3[j3];
            if (x) o = fma(a, xr[r], o);
            if (y) o = fma(b, yr[r], o);
            out[base + j] = o;
        }
    }
}

template <int N>
size_t fused_smem() { return sizeof(float2) * (size_t)N * N * (N + 1); }

// dynamic shared memory above the default 48 KB needs the kernel's opt-in
template <typename Kern>
int allow_smem(Kern kern, size_t bytes, const char *what)
{
    if (bytes <= 48 * 1024) return CS_OK;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return e == cudaSuccess ? CS_OK : cuda_error(e, what);
}

template <int N>
int forward_n(const Handle &hd, const double *f, int ncells, int grid_cells, cudaStream_t s)
{
    const float cf = (float)(pow(2.0 * M_PI, -1.5) * hd.g.dv * hd.g.dv * hd.g.dv);
    const unsigned blocks = (unsigned)(ngroups_of(std::max(ncells, grid_cells)) * kGroup);
    if (int rc = allow_smem(forward_fused_kernel<N>, fused_smem<N>(), "fused forward: shared-memory attribute")) return rc;
    forward_fused_kernel<N><<<blocks, kThreads<N>, fused_smem<N>(), s>>>(f, ncells, cf, (float2 *)hd.F);
    CS_LAUNCHED(1, s, "forward transform (fused)");
    return CS_OK;
}

template <int N>
int inverse_n(const Handle &hd, int ncells, double eps, int project, double a, const double *x, double b,
              const double *y, double c, double *out, const void *qh2, cudaStream_t s)
{
    Proj5 pj;
    for (int i = 0; i < 25; ++i) pj.ainv[i] = hd.cct_inv[i];
    // the scale of the last inverse pass, times the step factor c
    const float cic = (float)(c * pow(2.0 * M_PI, -1.5) * hd.g.dz * hd.g.dz * hd.g.dz / eps);
    if (int rc = allow_smem(inverse_project_kernel<N>, fused_smem<N>(), "fused inverse: shared-memory attribute"))
        return rc;
    inverse_project_kernel<N><<<ncells, kThreads<N>, fused_smem<N>(), s>>>(
        (const float2 *)hd.Qh, (const float2 *)qh2, cic, hd.g.dv, project, pj, a, x, b, y, out);
    CS_LAUNCHED(1, s, "inverse transform and projection (fused)");
    return CS_OK;
}

}  // namespace

bool fused_available(const Handle &hd)
{
    return hd.precision == CS_FP32 && (hd.g.N == 8 || hd.g.N == 12 || hd.g.N == 16 || hd.g.N == 24);
}

int launch_forward_fused(const Handle &hd, const double *f, int ncells, cudaStream_t s, int grid_cells)
{
    switch (hd.g.N) {
    case 8: return forward_n<8>(hd, f, ncells, grid_cells, s);
    case 12: return forward_n<12>(hd, f, ncells, grid_cells, s);
    case 16: return forward_n<16>(hd, f, ncells, grid_cells, s);
    case 24: return forward_n<24>(hd, f, ncells, grid_cells, s);
    default: return set_error(CS_ENOTSUP, "fused forward transform: unsupported N");
    }
}

int launch_inverse_project(const Handle &hd, int ncells, double eps, int project, double a, const double *x,
                           double b, const double *y, double c, double *out, const void *qh2, cudaStream_t s)
{
    switch (hd.g.N) {
    case 8: return inverse_n<8>(hd, ncells, eps, project, a, x, b, y, c, out, qh2, s);
    case 12: return inverse_n<12>(hd, ncells, eps, project, a, x, b, y, c, out, qh2, s);
    case 16: return inverse_n<16>(hd, ncells, eps, project, a, x, b, y, c, out, qh2, s);
    case 24: return inverse_n<24>(hd, ncells, eps, project, a, x, b, y, c, out, qh2, s);
    default: return set_error(CS_ENOTSUP, "fused inverse transform: unsupported N");
    }
}

}  // namespace cs
