// Whole-cell transforms for float handles with N in {8, 12, 16, 24, 32}.
// Up to N = 24 one cell's spectrum (N^3 complex floats, 32 KB at N = 16,
// 113 KB at N = 24) fits in one block's shared memory.  At N = 32 (256 KB) a
// cell takes a cluster of two blocks on two SMs: block r holds the v1-planes
// 16r .. 16r+15 (132 KB), the passes along axes 2 and 3 stay inside a block,
// and the pass along axis 1 reads and writes the partner's half through
// distributed shared memory; the projection's moments are summed over the
// pair the same way.
//
// forward_fused_kernel: one block per cell.  The cell's f is read once
// (contiguous), the three axis passes of the forward transform of Sec. 3.2,
//   fhat_k = (2 pi)^{-3/2} dv^3 sum_j f_j exp(-i zeta_k . v_j),
// run in shared memory, and fhat goes out in the 32-cell grouped layout the
// convolution reads.
//
// inverse_project_kernel: one block per cell.  Reads Qhat of the cell, runs
// the three
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
// 96th of a turn, which covers N = 8, 12, 16, 24, 32).  One thread owns one line, so
// the passes need no synchronisation inside a pass.
//
// Shared-memory layout of a block's planes: element (i1, i2, i3) at
// (p N + i2)(N + 1) + i3 in the block of rank i1 / PL, p = i1 mod PL (PL = N
// planes per block, or N/2 in a cluster pair); the +1 pad keeps the three
// line directions free of bank conflicts.
#include <algorithm>

#include <cooperative_groups.h>

#include "cs_internal.cuh"

namespace cs {

namespace {

// cos(2 pi e / 96) for e = 0 .. 24 (a quarter turn); other angles by symmetry
__host__ __device__ constexpr float cos96q(int e)
{
    constexpr float c[25] = {1.0f,         0.997858923f, 0.991444861f, 0.980785280f, 0.965925826f,
                             0.946930129f, 0.923879533f, 0.896872742f, 0.866025404f, 0.831469612f,
                             0.793353340f, 0.751839807f, 0.707106781f, 0.659345815f, 0.608761429f,
                             0.555570233f, 0.5f,         0.442288690f, 0.382683432f, 0.321439465f,
                             0.258819045f, 0.195090322f, 0.130526192f, 0.065403129f, 0.0f};
    return c[e];
}

__host__ __device__ constexpr float cos96(int e)
{
    return e <= 24 ? cos96q(e) : e <= 48 ? -cos96q(48 - e) : e <= 72 ? -cos96q(e - 48) : cos96q(96 - e);
}

__host__ __device__ constexpr float sin96(int e) { return cos96((e + 72) % 96); }  // sin t = cos(t - quarter turn)

// x * w^m with w = exp(-2 pi i / R) (forward) or exp(+2 pi i / R) (inverse),
// m a compile-time value after unrolling; quarter turns are exact swaps
template <int R, bool INV>
__device__ __forceinline__ float2 rot(float2 x, int m)
{
    static_assert(96 % R == 0, "twiddles in 96ths of a turn");
    const int e = (m % R) * (96 / R);
    if (e == 0) return x;
    if (e == 48) return make_float2(-x.x, -x.y);
    if (e == 24) return INV ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
    if (e == 72) return INV ? make_float2(x.y, -x.x) : make_float2(-x.y, x.x);
    const float c = cos96(e), s = INV ? sin96(e) : -sin96(e);
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

// Blocks per cell CL (a cluster pair at N = 32, where a cell does not fit
// one SM; splitting smaller cells over a pair as well measured slower, even
// at 128 cells where one block per cell leaves SMs idle), v1-planes per
// block, lines a block transforms per pass (one per thread, rounded up to
// whole warps for the shuffled reductions: 64, 160, 256, 576, 512 for
// N = 8, 12, 16, 24, 32)
template <int N>
constexpr int kCL = N == 32 ? 2 : 1;
template <int N, int CL>
constexpr int kPL = N / CL;
template <int N, int CL>
constexpr int kLines = kPL<N, CL> * N;
template <int N, int CL>
constexpr int kThreads = (kLines<N, CL> + 31) / 32 * 32 < 64 ? 64 : (kLines<N, CL> + 31) / 32 * 32;

// loops over a block's kPts points run kPer rounds of the block, in chunks
// of kChunk rounds unrolled with every global load of a chunk issued before
// its first use (one chunk up to 16 rounds; chunks of 8 at N = 24 and 32,
// which keeps the registers of a 576- or 512-thread block within its share)
template <int N, int CL>
constexpr int kPts = kPL<N, CL> * N * N;
template <int N, int CL>
constexpr int kPer = (kPts<N, CL> + kThreads<N, CL> - 1) / kThreads<N, CL>;
template <int N, int CL>
constexpr int kChunk = kPer<N, CL> <= 16 ? kPer<N, CL> : 8;

struct Proj5 {
    double ainv[25];
};

namespace cg = cooperative_groups;

// every block of the cell's cluster has finished its accesses to shared memory
// (its own and, through the cluster, the partner's) before any goes on
template <int CL>
__device__ __forceinline__ void cell_sync()
{
    if constexpr (CL == 2)
        cg::this_cluster().sync();
    else
        __syncthreads();
}

template <int CL>
__device__ __forceinline__ int cell_rank()
{
    if constexpr (CL == 2)
        return (int)cg::this_cluster().block_rank();
    else
        return 0;
}

// the shared array X of every block of the cell, by rank
template <int CL>
__device__ __forceinline__ void cell_arrays(float2 *X, int rank, float2 *(&Xr)[CL])
{
    if constexpr (CL == 2) {
        float2 *peer = cg::this_cluster().map_shared_rank(X, rank ^ 1);
        Xr[rank] = X;
        Xr[rank ^ 1] = peer;
    } else {
        Xr[0] = X;
    }
}

// the transform along axis 1 of line l of block `rank`: (i2, i3) =
// (rank PL + l / N, l mod N); element i1 sits in block i1 / PL
template <int N, bool INV, int CL>
__device__ __forceinline__ void axis1_transform(float2 *const (&Xr)[CL], int rank, int l, float scale)
{
    constexpr int P = N + 1, PL = kPL<N, CL>;
    const int i2 = rank * PL + l / N, i3 = l % N;
    float2 v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const float2 t = Xr[j / PL][((j % PL) * N + i2) * P + i3];
        v[j] = (j & 1) ? make_float2(-t.x, -t.y) : t;
    }
    fft<N, INV>(v);
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const float sk = (k & 1) ? -scale : scale;
        Xr[k / PL][((k % PL) * N + i2) * P + i3] = make_float2(sk * v[k].x, sk * v[k].y);
    }
}

template <int N, int CL>
__global__ void __launch_bounds__(kThreads<N, CL>) forward_fused_kernel(const double *__restrict__ f, int ncells,
                                                                        float cf, float2 *__restrict__ F)
{
    constexpr int M = N * N * N, P = N + 1, NT = kThreads<N, CL>, LINES = kLines<N, CL>, PTS = kPts<N, CL>;
    constexpr int PER = kPer<N, CL>, CHUNK = kChunk<N, CL>;
    extern __shared__ float2 X[];  // [PL*N][P]
    const int cell = blockIdx.x / CL;
    const int rank = cell_rank<CL>();
    const int tid = threadIdx.x;
    const bool real = cell < ncells;
    const size_t gbase = (size_t)cell * M + (size_t)rank * PTS;  // the block's planes in f
    static_assert(PER % CHUNK == 0, "whole chunks");
    for (int r0 = 0; r0 < PER; r0 += CHUNK) {
        double fr[CHUNK];
#pragma unroll
        for (int r = 0; r < CHUNK; ++r) {
            const int j = (r0 + r) * NT + tid;
            fr[r] = (real && j < PTS) ? f[gbase + j] : 0.0;
        }
#pragma unroll
        for (int r = 0; r < CHUNK; ++r) {
            const int j = (r0 + r) * NT + tid;
            if (j < PTS) X[(j / N) * P + j % N] = make_float2((float)fr[r], 0.f);
        }
    }
    __syncthreads();
    const int l = tid;
    if (l < LINES) line_transform<N, false>(X, l * P, 1, 1.f);  // axis 3
    __syncthreads();
    if (l < LINES) line_transform<N, false>(X, (l / N) * N * P + l % N, P, 1.f);  // axis 2
    cell_sync<CL>();
    {
        float2 *Xr[CL];
        cell_arrays<CL>(X, rank, Xr);
        if (l < LINES) axis1_transform<N, false, CL>(Xr, rank, l, cf);  // axis 1
    }
    cell_sync<CL>();
    const int g = cell / kGroup, lane = cell % kGroup;
    const size_t fbase = (size_t)g * M + (size_t)rank * PTS;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int k = r * NT + tid;
        if (k < PTS) F[(fbase + k) * kGroup + lane] = X[(k / N) * P + k % N];
    }
}

template <int N, int CL>
__global__ void __launch_bounds__(kThreads<N, CL>) inverse_project_kernel(
    const float2 *__restrict__ Qh, float cic, double dv, int project, Proj5 pj, double a, const double *x, double b,
    const double *y, double *out, float2 *__restrict__ Fnext, float cf)
{
    constexpr int M = N * N * N, P = N + 1, LINES = kLines<N, CL>, PL = kPL<N, CL>, PTS = kPts<N, CL>, H = N / 2;
    constexpr int NT = kThreads<N, CL>, NW = NT / 32, PER = kPer<N, CL>, CHUNK = kChunk<N, CL>;
    static_assert(NT % 32 == 0, "whole warps");
    extern __shared__ float2 X[];  // [PL*N][P]; after the transform, reused as double q = c Qt
    __shared__ double vax[N], vsq[N], cv3[N], lbase[LINES];
    __shared__ double red[5][NW];
    __shared__ double ycoef[5], mom_s[5], part[5];
    const int cell = blockIdx.x / CL;
    const int rank = cell_rank<CL>();
    const int g = cell / kGroup, lane = cell % kGroup;
    const int tid = threadIdx.x;
    if (tid < N) {
        vax[tid] = dv * (tid - H);
        vsq[tid] = vax[tid] * vax[tid];
    }
    const size_t fbase = (size_t)g * M + (size_t)rank * PTS;  // the block's planes in Qh
    for (int r0 = 0; r0 < PER; r0 += CHUNK) {
        float2 qa[CHUNK];
#pragma unroll
        for (int r = 0; r < CHUNK; ++r) {
            const int k = (r0 + r) * NT + tid;
            qa[r] = Qh[(fbase + (k < PTS ? k : 0)) * kGroup + lane];
        }
#pragma unroll
        for (int r = 0; r < CHUNK; ++r) {
            const int k = (r0 + r) * NT + tid;
            if (k < PTS) X[(k / N) * P + k % N] = qa[r];
        }
    }
    cell_sync<CL>();
    const int l = tid;
    {
        float2 *Xr[CL];
        cell_arrays<CL>(X, rank, Xr);
        if (l < LINES) axis1_transform<N, true, CL>(Xr, rank, l, 1.f);  // axis 1
    }
    cell_sync<CL>();
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
        // moments of the line (j1, j2) = (rank PL + l / N, l mod N): S0 = sum q,
        // S3 = sum v3 q, S33 = sum v3^2 q
        double s0 = 0, s3 = 0, s33 = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const double qq = (double)(((k & 1) ? -cic : cic) * v[k].x);
            Qd[l * P + k] = qq;
            s0 += qq;
            s3 = fma(vax[k], qq, s3);
            s33 = fma(vsq[k], qq, s33);
        }
        const int j1 = rank * PL + l / N, j2 = l % N;
        m[0] = s0;
        m[1] = vax[j1] * s0;
        m[2] = vax[j2] * s0;
        m[3] = s3;
        m[4] = fma(vsq[j1] + vsq[j2], s0, s33);
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
    // moments (thread i sums moment i over the warps, then over the cluster's
    // blocks in rank order), then y = (C C^T)^{-1} C q (thread i takes row
    // i); every block of the cell gets the same doubles
    const double w3 = dv * dv * dv;
    if (tid < 5) {
        double t = 0;
        if (project)
            for (int k = 0; k < NW; ++k) t += red[tid][k];
        part[tid] = t;
    }
    if constexpr (CL == 2) {
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        if (tid < 5) {
            const double *p0 = cl.map_shared_rank(part, 0), *p1 = cl.map_shared_rank(part, 1);
            mom_s[tid] = w3 * (p0[tid] + p1[tid]);
        }
        cl.sync();  // both blocks have read the partner's partial sums
    } else {
        if (tid < 5) mom_s[tid] = w3 * part[tid];
        __syncthreads();
    }
    if (tid < 5) {
        double s = 0;
        if (project)
            for (int k = 0; k < 5; ++k) s += pj.ainv[5 * tid + k] * mom_s[k];
        ycoef[tid] = w3 * s;  // C^T y = w3 (1, v1, v2, v3, |v|^2) . y
    }
    __syncthreads();
    const double y0 = ycoef[0], y1 = ycoef[1], y2 = ycoef[2], y3 = ycoef[3], y4 = ycoef[4];
    // correction C^T y at (v1, v2, v3) = lbase(v1, v2) + cv3(v3), for the block's lines
    for (int i = tid; i < LINES; i += NT) {
        const int j1 = rank * PL + i / N, j2 = i % N;
        lbase[i] = fma(y4, vsq[j1] + vsq[j2], fma(y2, vax[j2], fma(y1, vax[j1], y0)));
    }
    if (tid < N) cv3[tid] = vax[tid] * fma(y4, vax[tid], y3);
    __syncthreads();
    const size_t base = (size_t)cell * M + (size_t)rank * PTS;
    // x and y may alias out (same index, same thread only): a chunk's loads
    // come before its stores
    for (int r0 = 0; r0 < PER; r0 += CHUNK) {
        double xr[CHUNK], yr[CHUNK];
#pragma unroll
        for (int r = 0; r < CHUNK; ++r) {
            const int j = (r0 + r) * NT + tid;
            xr[r] = (x && j < PTS) ? x[base + j] : 0.0;
            yr[r] = (y && j < PTS) ? y[base + j] : 0.0;
        }
#pragma unroll
        for (int r = 0; r < CHUNK; ++r) {
            const int j = (r0 + r) * NT + tid;
            if (j >= PTS) break;
            const int jl = j / N, j3 = j % N;
            double o = Qd[jl * P + j3];
            if (project) o -= lbase[jl] + cv3[j3];
            if (x) o = fma(a, xr[r], o);
            if (y) o = fma(b, yr[r], o);
            out[base + j] = o;
            // the slot just read, reused for the forward transform of out (same thread)
            if (Fnext) X[jl * P + j3] = make_float2((float)o, 0.f);
        }
    }
    if constexpr (CL == 1) {
        // the forward transform of out, as forward_fused_kernel computes it from
        // the same values (the next Heun evaluation's input; padding lanes of
        // the last group keep the zeros the previous forward wrote)
        if (Fnext) {
            __syncthreads();
            if (l < LINES) line_transform<N, false>(X, l * P, 1, 1.f);  // axis 3
            __syncthreads();
            if (l < LINES) line_transform<N, false>(X, (l / N) * N * P + l % N, P, 1.f);  // axis 2
            __syncthreads();
            if (l < LINES) line_transform<N, false>(X, (l / N) * P + l % N, N * P, cf);  // axis 1
            __syncthreads();
#pragma unroll
            for (int r = 0; r < PER; ++r) {
                const int k = r * NT + tid;
                if (k < PTS) Fnext[((size_t)g * M + k) * kGroup + lane] = X[(k / N) * P + k % N];
            }
        }
    }
}

template <int N, int CL>
size_t fused_smem() { return sizeof(float2) * (size_t)kPL<N, CL> * N * (N + 1); }

// dynamic shared memory above the default 48 KB needs the kernel's opt-in
template <typename Kern>
int allow_smem(Kern kern, size_t bytes, const char *what)
{
    if (bytes <= 48 * 1024) return CS_OK;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return e == cudaSuccess ? CS_OK : cuda_error(e, what);
}

// launch with CL blocks per cell, as a cluster when there are two
template <int N, int CL, typename... Args>
cudaError_t launch_cells(void (*kern)(Args...), unsigned cells, cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cells * CL);
    cfg.blockDim = dim3(kThreads<N, CL>);
    cfg.dynamicSmemBytes = fused_smem<N, CL>();
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = CL > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <int N, int CL>
int forward_cl(const Handle &hd, const double *f, int ncells, unsigned cells, float cf, cudaStream_t s)
{
    if (int rc = allow_smem(forward_fused_kernel<N, CL>, fused_smem<N, CL>(), "fused forward: shared-memory attribute"))
        return rc;
    cudaError_t e = launch_cells<N, CL>(forward_fused_kernel<N, CL>, cells, s, f, ncells, cf, (float2 *)hd.F);
    if (e != cudaSuccess) return cuda_error(e, "fused forward transform launch");
    CS_LAUNCHED(1, s, "forward transform (fused)");
    return CS_OK;
}

template <int N>
int forward_n(const Handle &hd, const double *f, int ncells, int grid_cells, cudaStream_t s)
{
    const float cf = (float)(pow(2.0 * M_PI, -1.5) * hd.g.dv * hd.g.dv * hd.g.dv);
    const unsigned cells = (unsigned)(ngroups_of(std::max(ncells, grid_cells)) * kGroup);
    return forward_cl<N, kCL<N>>(hd, f, ncells, cells, cf, s);
}

template <int N, int CL>
int inverse_cl(const Handle &hd, int ncells, float cic, int project, const Proj5 &pj, double a, const double *x,
               double b, const double *y, double *out, void *fnext, cudaStream_t s)
{
    if (int rc = allow_smem(inverse_project_kernel<N, CL>, fused_smem<N, CL>(), "fused inverse: shared-memory attribute"))
        return rc;
    const float cf = (float)(pow(2.0 * M_PI, -1.5) * hd.g.dv * hd.g.dv * hd.g.dv);
    cudaError_t e = launch_cells<N, CL>(inverse_project_kernel<N, CL>, (unsigned)ncells, s, (const float2 *)hd.Qh,
                                        cic, hd.g.dv, project, pj, a, x, b, y, out,
                                        CL == 1 ? (float2 *)fnext : (float2 *)nullptr, cf);
    if (e != cudaSuccess) return cuda_error(e, "fused inverse transform launch");
    CS_LAUNCHED(1, s, "inverse transform and projection (fused)");
    return CS_OK;
}

template <int N>
int inverse_n(const Handle &hd, int ncells, double eps, int project, double a, const double *x, double b,
              const double *y, double c, double *out, void *fnext, cudaStream_t s)
{
    Proj5 pj;
    for (int i = 0; i < 25; ++i) pj.ainv[i] = hd.cct_inv[i];
    // the scale of the last inverse pass, times the step factor c
    const float cic = (float)(c * pow(2.0 * M_PI, -1.5) * hd.g.dz * hd.g.dz * hd.g.dz / eps);
    return inverse_cl<N, kCL<N>>(hd, ncells, cic, project, pj, a, x, b, y, out, fnext, s);
}

}  // namespace

bool fused_forward_next(const Handle &hd)
{
    return fused_available(hd) && hd.g.N != 32 && hd.tune_fwd_next != 2;
}

bool fused_available(const Handle &hd)
{
    const int N = hd.g.N;
    return hd.precision == CS_FP32 && (N == 8 || N == 12 || N == 16 || N == 24 || N == 32);
}

int launch_forward_fused(const Handle &hd, const double *f, int ncells, cudaStream_t s, int grid_cells)
{
    switch (hd.g.N) {
    case 8: return forward_n<8>(hd, f, ncells, grid_cells, s);
    case 12: return forward_n<12>(hd, f, ncells, grid_cells, s);
    case 16: return forward_n<16>(hd, f, ncells, grid_cells, s);
    case 24: return forward_n<24>(hd, f, ncells, grid_cells, s);
    case 32: return forward_n<32>(hd, f, ncells, grid_cells, s);
    default: return set_error(CS_ENOTSUP, "fused forward transform: unsupported N");
    }
}

int launch_inverse_project(const Handle &hd, int ncells, double eps, int project, double a, const double *x,
                           double b, const double *y, double c, double *out, cudaStream_t s, void *fnext)
{
    if (fnext && !fused_forward_next(hd)) return set_error(CS_ENOTSUP, "fused inverse: no forward transform at this N");
    switch (hd.g.N) {
    case 8: return inverse_n<8>(hd, ncells, eps, project, a, x, b, y, c, out, fnext, s);
    case 12: return inverse_n<12>(hd, ncells, eps, project, a, x, b, y, c, out, fnext, s);
    case 16: return inverse_n<16>(hd, ncells, eps, project, a, x, b, y, c, out, fnext, s);
    case 24: return inverse_n<24>(hd, ncells, eps, project, a, x, b, y, c, out, fnext, s);
    case 32: return inverse_n<32>(hd, ncells, eps, project, a, x, b, y, c, out, fnext, s);
    default: return set_error(CS_ENOTSUP, "fused inverse transform: unsupported N");
    }
}

}  // namespace cs
